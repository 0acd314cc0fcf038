/*
 * cfdem.h -- C ABI of the GB300 CFD-DEM coupling library.
 *
 * One coupling step of unresolved CFD-DEM on a Q_k (k = 1..3) Lagrange
 * hexahedral mesh, as stated in "Towards High-Order CFD-DEM: Development and
 * Validation" (arXiv 2211.01185):
 *   - void fraction from particle positions and radii (Eq. void_fraction,
 *     Sec. 2.1), quadrature-centred (QCM) or particle-centroid (PCM);
 *   - its smoothed L2 projection onto the nodal Q_k space, with smoothing
 *     length L^2 (the "void fraction smoothing factor" of Tables setup1,
 *     setup2 and setup4): (M + L^2 K) eps_h = b;
 *   - per-particle drag, buoyancy and pressure-gradient forces (Sec. 2.3.2,
 *     Eqs. drag, beta, the Dallavalle and Di Felice C_D, buoyancy and
 *     undisturbed-flow forces) and the fluid source term F_pf (Eqs. fb, fa).
 *
 * Conventions shared by every call:
 *   - Pointers named *_dev are device pointers on the context's device; the
 *     caller owns them.  Arrays are C-contiguous FP64 unless stated:
 *     positions x[n][3], radii r[n], particle velocities u_p[n][3], nodal
 *     velocities u[n_nodes][3], nodal pressure p[n_pnodes].
 *   - Element e = ex + Nx (ey + Ny ez); quadrature point q = qx + nq (qy + nq
 *     qz) with nq = k + 1 Gauss-Legendre points per axis; node n = ix + (Nx k
 *     + 1)(iy + (Ny k + 1) iz) with GLL points inside each element.  The
 *     pressure space is Q_kp on the same elements (kp = pressure_degree).
 *   - Every call is ordered on the context's CUDA stream and returns without
 *     synchronising.  Errors found on the device (a particle outside the
 *     mesh, an unconverged solve) are reported by the next cfdem_synchronize
 *     or cfdem_get_stats.  No call aborts the process or traps the GPU.
 *   - The context owns its scratch memory and grows it on demand; a call that
 *     needs to grow it must not be inside stream capture.
 *   - Results of the FP64 path match the FP64 CPU oracle within 1e-10
 *     (relative to max(|b_i|, 1e-3 max|b|)); indices (element, bin, sort
 *     order, neighbour counts) are bit-exact.  The mixed path matches within
 *     1e-5.
 */
#ifndef CFDEM_H
#define CFDEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cfdem_ctx *cfdem_t;

typedef enum {
    CFDEM_OK = 0,
    CFDEM_EINVAL = -1,          /* bad argument; nothing was launched */
    CFDEM_OUT_OF_DOMAIN = -2,   /* a particle centre lies outside the mesh */
    CFDEM_NOT_CONVERGED = -3,   /* CG stopped at cg_maxit; last iterate kept */
    CFDEM_ENOMEM = -4,          /* device allocation failed */
    CFDEM_ECUDA = -5,           /* a CUDA runtime call failed */
    CFDEM_ESTATE = -6,          /* call needs set_mesh / a previous stage */
    CFDEM_ECAPACITY = -7        /* a fixed per-particle capacity was exceeded */
} cfdem_status;

/* Physical and numerical parameters.  cfdem_params_default fills them. */
typedef struct {
    double rho_f;          /* fluid density [kg/m^3] */
    double mu_f;           /* fluid dynamic viscosity [Pa s] */
    double g[3];           /* gravity [m/s^2]; buoyancy f_B = -rho_f V_p g */
    int scheme;            /* 0 = QCM (quadrature-centred), 1 = PCM */
    double qcm_radius;     /* averaging-sphere radius R; 0 => (3 V_e / 4 pi)^(1/3) */
    double l2_smoothing;   /* L^2 [m^2]; 0 => plain L2 (mass) projection */
    int drag_model;        /* closure of Sec. 2.3.2: 0 = Di Felice, 1 = Dallavalle,
                              2 = Rong, 3 = Koch-Hill, 4 = Gidaspow (Ergun below
                              eps 0.8, Wen-Yu above), 5 = Beetstra */
    int vans_model;        /* 0 = model A (F_pf from drag), 1 = model B (drag + grad p) */
    int beta_over_eps;     /* 1 => beta_B = beta_A / eps (Eq. beta) */
    int precision;         /* 0 = FP64, 1 = mixed (FP32 work, FP64 refinement) */
    double cg_rtol;        /* stop when ||b - A x||_2 <= cg_rtol ||b||_2 */
    int cg_maxit;          /* iteration cap of the solve */
    double eps_floor;      /* closures use eps_c = min(max(eps, eps_floor), 1) */
    int pressure_degree;   /* kp; 0 => max(1, k - 1) */
    double max_radius;     /* hint for the bin size (largest particle radius); 0 => R */
    double bin_edge;       /* bin edge [m]; 0 => R + max_radius */
    int cg_precond;        /* 0 = Jacobi, 1 = fast diagonalisation (exact inverse of the
                              Kronecker-sum operator, applied in FP32; default) */
    int shear_force;       /* 1 => add the shear force -V_p div tau (Sec. 2.3.2,
                              undisturbed-flow forces; tau the deviatoric stress of
                              Eq. (stress), second derivatives of the Q_k velocity
                              at the particle) to f, and for model B to the fluid
                              source; default 0 */
    int fluid_drag;        /* drag on the fluid side: 0 = explicit, F_pf,e = -(1/V_e)
                              sum_{i in e} f_D,i per element (Eqs. fa/fb); 1 = the
                              fluid-side form of Sec. 2.3.2, F_pf(x_q) = -beta_e
                              (u_f(x_q) - u_p,avg,e) with beta_e = (1/V_e) sum_i beta_i
                              and u_p,avg,e the plain mean particle velocity in e
                              (F_q then varies over the element; F_elem is its Gauss
                              average; see cfdem_fluid_drag_coefficients); default 0 */
    int qcm_conserve;      /* 1 => volume-conserving QCM: each particle's lens volumes
                              are scaled by c_i = V_p,i / S_i, S_i = sum_q w_q |J|
                              V(R, r_i, d_iq) / V_R the volume the plain sum puts on the
                              mesh, so that sum_q w_q |J| (1 - eps_q) = sum_i V_p,i also
                              where averaging spheres cross the walls; not supported by
                              cfdem_adjoint (CFDEM_EINVAL); default 0 */
    int autotune;          /* 1 => the first eager step of a new signature (mesh, degree,
                              precision, particle count within a factor of two, largest
                              radius) times a few bin edges of the QCM's particle bins
                              (fractions of R + max_radius, and h / m so that bins nest in
                              elements) and the three tile shapes of the projection
                              operator, and keeps the fastest for the context (and for
                              later contexts of the same signature in the process).
                              Results do not depend on the choice beyond the order of
                              floating-point sums (neighbour sets are the same).  The
                              timing synchronises the stream, once per signature; nothing
                              is timed while the stream is being captured.  0 => bins of
                              edge R + max_radius and the shape of a static cost model.
                              bin_edge > 0 fixes the bins either way.  Default 1. */
} cfdem_params;

/* Counters of the last calls on a context. */
typedef struct {
    int64_t first_bad_particle;   /* -1 or the lowest index found outside the mesh */
    int32_t cg_iterations;        /* total (inner) iterations of the last solve */
    int32_t cg_outer;             /* refinement steps of the last mixed solve */
    double cg_relres;             /* ||b - A x|| / ||b|| at exit */
    int32_t converged;            /* 1 if the last solve met cg_rtol */
    int32_t nb[3];                /* bins per axis */
    double bin_edge[3];           /* bin edges [m] */
    double qcm_radius;            /* resolved averaging radius [m] */
    int64_t n_elem, n_qp, n_nodes, n_pnodes;
    /* with cfdem_set_timing(ctx, 1): device time [ms] and calls per stage
     * since the last cfdem_set_timing: 0 locate+bin (a1-a2), 1 void fraction
     * kernel (a3), 2 right-hand side (a4), 3 whole solve (a5), 4 forces (a6),
     * 5 fluid source (a7), 6 FP32 operator launches, 7 FP64 operator
     * launches */
    double stage_ms[8];
    int64_t stage_calls[8];
    int32_t timer_overflow;       /* 1 if more than 1024 pairs per stage were asked */
    int64_t kernel_launches;      /* kernels launched by the library since set_timing */
    int32_t precond;              /* preconditioner in use: 0 Jacobi, 1 FDM */
    int32_t tile_shape;           /* operator tile in use: 0 16x8x8, 1 22x13x4, 2 25x15x4 nodes */
    int32_t tuned;                /* bit 0: bins chosen by timing, bit 1: tile shape chosen by
                                     timing (autotune) */
    double tune_ms;               /* host time spent timing candidates in this context */
    int32_t fdm_tile;             /* register tile of the FDM slab transforms, 10 rows + columns
                                     (44 = 4 x 4; chosen by timing when the plan is built), 0
                                     without the slab form */
} cfdem_stats;

/* Create a context on CUDA device `device`, ordering all work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Returns CFDEM_ECUDA if the device cannot be used. */
cfdem_status cfdem_create(cfdem_t *out, int device, void *stream);

/* Free the context and all scratch memory it owns.  NULL is accepted. */
cfdem_status cfdem_destroy(cfdem_t ctx);

/* Fill *p with the defaults: gas (rho_f 1.2, mu_f 1.8e-5), g = (0,0,-9.81),
 * QCM, Di Felice, model A, FP64, cg_rtol 1e-13, cg_maxit 2000, eps_floor
 * 0.05, FDM preconditioner, everything else 0 (resolved from the mesh). */
void cfdem_params_default(cfdem_params *p);

/* Mesh: the axis-aligned box [origin, origin + extent] cut into n_el[0] x
 * n_el[1] x n_el[2] equal hexahedra carrying Q_degree (degree 1..3).  The
 * paper couples both phases on this one mesh (Sec. 2.3).  Host pointers. */
cfdem_status cfdem_set_mesh(cfdem_t ctx, const double origin[3], const double extent[3],
                            const int n_el[3], int degree);

/* Parameters (host struct, copied).  Resolves R, kp and the bin grid. */
cfdem_status cfdem_set_params(cfdem_t ctx, const cfdem_params *p);

/* The resolved parameters (qcm_radius, pressure_degree, bin_edge filled). */
cfdem_status cfdem_get_params(cfdem_t ctx, cfdem_params *p);

/* Step a1 -- element location (Sec. 2.3: particles live on the fluid mesh).
 * elem_dev[n] (int32) = element of each centre: per axis floor((x - x0)/h)
 * with IEEE division, clamped to [0, N-1] (a centre on an interior face
 * belongs to the upper element); xi_dev[n][3] = reference coordinates
 * (x - x0)/h - e_axis.  Either output may be NULL.  A centre outside the box
 * by more than 1e-12 of its extent gets elem = -1 and sets
 * CFDEM_OUT_OF_DOMAIN. */
cfdem_status cfdem_locate(cfdem_t ctx, int64_t n, const double *x_dev, int32_t *elem_dev,
                          double *xi_dev);

/* Step a2 -- stable counting sort of the particles into the context's bin
 * grid (bin = per-axis floor((x - x0)/b), clamped; bx fastest).  Outputs
 * (device, optional): bin_start_dev[nbins + 1] exclusive prefix of the bin
 * counts, perm_dev[n] particle ids in bin order, ascending inside a bin. */
cfdem_status cfdem_bin(cfdem_t ctx, int64_t n, const double *x_dev, int32_t *bin_start_dev,
                       int32_t *perm_dev);

/* Steps a1-a3 -- void fraction at every quadrature point, eps_q_dev[E][Q].
 * QCM: eps_q = 1 - sum_i V_lens(R, r_i, |x_q - x_i|) / (4/3 pi R^3) over the
 * particles with |x_q - x_i|^2 < (R + r_i)^2 (a reading of the deferred
 * void-fraction scheme; Eq. void_fraction gives its particle-centroid
 * limit).  PCM: eps_e = (V_e - sum_{i in e} V_p,i) / V_e (Eq.
 * void_fraction), copied to all Q points.  eps_q_dev may be NULL: the
 * result is then kept inside the context for cfdem_project.  nb_count_dev
 * [E][Q] (int32) and nb_idsum_dev [E][Q] (int64), optional, receive the
 * QCM neighbour count and the sum of neighbour ids per point. */
cfdem_status cfdem_void_fraction(cfdem_t ctx, int64_t n, const double *x_dev,
                                 const double *r_dev, double *eps_q_dev, int32_t *nb_count_dev,
                                 int64_t *nb_idsum_dev);

/* Step a4 -- projection right-hand side b_j = sum_e sum_q phi_j(x_q) w_q
 * |J_e| eps_q from eps_q_dev[E][Q] (NULL = the context's last void
 * fraction); b_dev[n_nodes]. */
cfdem_status cfdem_project_rhs(cfdem_t ctx, const double *eps_q_dev, double *b_dev);

/* The projection operator y = (M + L^2 K) x on nodal vectors (device,
 * n_nodes), matrix-free and sum-factorised. */
cfdem_status cfdem_apply(cfdem_t ctx, const double *x_dev, double *y_dev);

/* Steps a4-a5 -- smoothed L2 projection: solves (M + L^2 K) eps_h = b by
 * preconditioned CG.  FP64: CG in FP64.  Mixed: CG with double-float (FP32
 * pair) iterate, residual and operator and the FP32 preconditioner as inner
 * solver, or, without the fast-diagonalisation preconditioner, FP32 CG
 * inside FP64 iterative refinement.  Preconditioner: Jacobi or fast
 * diagonalisation (cg_precond).  eps_q_dev: NULL = the context's last void
 * fraction.  eps_nodal_dev[n_nodes]: start vector on entry, solution on exit.
 * The iteration count and relative residual go to cfdem_get_stats.
 * While the context's stream is being captured into a CUDA graph the CG
 * loop becomes a conditional (while) node of that graph that iterates on the
 * device until convergence or cg_maxit; the statistics of a replay are read
 * by the next cfdem_synchronize / cfdem_get_stats.  Capture requires the
 * stage timers off and, for the mixed path, the fast-diagonalisation
 * preconditioner (else CFDEM_ESTATE). */
cfdem_status cfdem_project(cfdem_t ctx, const double *eps_q_dev, double *eps_nodal_dev);

/* Steps a6-a7 -- particle forces and fluid source.  Per particle i: u_f,
 * eps (Q_k) and grad p (Q_kp) interpolated at x_i; eps_c clamped to
 * [eps_floor, 1] for the closures; Re_p = rho_f eps_c |u_f - u_p| d_p /
 * mu_f; f_D = beta_i (u_f - u_p) with the closure of drag_model (Sec.
 * 2.3.2), divided by eps_c if beta_over_eps; f_B = -rho_f V_p g; f_gradp =
 * -V_p grad p; f_shear = -V_p div tau if shear_force; f = f_D + f_B +
 * f_gradp (+ f_shear).  Fluid source per element F_e = -(1/V_e) sum_{i in
 * e} S_i with S_i = f_D (model A) or f_D + f_gradp (+ f_shear) (model B);
 * with fluid_drag = 1 the drag part is -beta_e (u_f(x_q) - u_p,avg,e) at
 * each quadrature point instead.  Outputs (device): f_dev[n][3] required;
 * f_drag_dev [n][3], F_elem_dev[E][3] and F_q_dev[E][Q][3] (the source at
 * every quadrature point) optional. */
cfdem_status cfdem_forces(cfdem_t ctx, int64_t n, const double *x_dev, const double *r_dev,
                          const double *u_p_dev, const double *u_nodal_dev,
                          const double *p_nodal_dev, const double *eps_nodal_dev,
                          double *f_dev, double *f_drag_dev, double *F_elem_dev,
                          double *F_q_dev);

/* The per-element coefficients of the fluid-side drag (fluid_drag = 1,
 * Sec. 2.3.2) from the last cfdem_forces / cfdem_coupling_step on this
 * context: beta_e[E] = (1/V_e) sum_{i in e} beta_i, beta_i the drag
 * coefficient of particle i (f_D,i = beta_i (u_f(x_i) - u_p,i)), and
 * up_avg[E][3] the mean velocity of the particles in e (0 in an empty
 * element), for a fluid solver that treats -beta_e (u_f - u_p,avg) in its
 * own (implicit) assembly.  Device pointers; either may be NULL.  Stream
 * ordered.  CFDEM_ESTATE if no forces call with fluid_drag = 1 ran since the
 * mesh was set. */
cfdem_status cfdem_fluid_drag_coefficients(cfdem_t ctx, double *beta_e, double *up_avg);

/* Steps a1-a7 in one call: void fraction, projection (eps_nodal_dev is the
 * start vector and receives eps_h), forces and fluid source.  Outputs as in
 * cfdem_forces. */
cfdem_status cfdem_coupling_step(cfdem_t ctx, int64_t n, const double *x_dev,
                                 const double *r_dev, const double *u_p_dev,
                                 const double *u_nodal_dev, const double *p_nodal_dev,
                                 double *eps_nodal_dev, double *f_dev, double *f_drag_dev,
                                 double *F_elem_dev, double *F_q_dev);

/* Adjoint of the coupling step (no counterpart in the paper: the
 * derivative of a loss J of the step's outputs with respect to its inputs,
 * for sensitivity studies and gradient-based calibration).  Given the
 * gradients of J with respect to the forces f (g_f_dev[n][3]), the drag
 * forces f_D (g_fdrag_dev[n][3]) and the projected void fraction eps_h
 * (g_eps_dev[n_nodes]) -- each NULL if J does not depend on it -- and the
 * forward step's inputs with its eps_nodal_dev (eps_h of that step), writes
 * dJ/dx (dJdx_dev[n][3]) and, if not NULL, dJ/du_nodal (dJdu_dev
 * [n_nodes][3]), by reverse-mode differentiation through the force closures
 * (forward-mode duals for their 3 x 4 Jacobian), the interpolations, the
 * projection (one more CG solve with the same operator, which is symmetric)
 * and the quadrature-centred void fraction (dV_lens/dd = -pi a^2, a the
 * radius of the circle where particle and averaging sphere meet).  The
 * particle-centroid void fraction is piecewise constant in x and adds
 * nothing; the fluid source is not an output of this derivative.  Precision
 * follows the context (mixed: closure Jacobian in FP32).  The CG statistics
 * of the adjoint solve replace those of the forward solve in
 * cfdem_get_stats. */
cfdem_status cfdem_adjoint(cfdem_t ctx, int64_t n, const double *x_dev, const double *r_dev,
                           const double *u_p_dev, const double *u_nodal_dev,
                           const double *p_nodal_dev, const double *eps_nodal_dev,
                           const double *g_f_dev, const double *g_fdrag_dev,
                           const double *g_eps_dev, double *dJdx_dev, double *dJdu_dev);

/* y = M x with M the consistent mass matrix of the nodal Q_k space (the
 * operator of cfdem_apply without the smoothing term), e.g. for the
 * gradient M eps_h / ||eps_h||_M of the L2 norm ||eps_h||_M. */
cfdem_status cfdem_mass_apply(cfdem_t ctx, const double *x_dev, double *y_dev);

/* ---- Batched ensemble of independent beds ------------------------------
 * An array of beds, each with its own mesh, degree, parameters and
 * particles, advanced by one coupling step each in one call (the many small
 * problems of a parameter study or an ensemble, which one at a time leave
 * most of the GPU idle).  The batch owns one context per bed, each with its
 * own stream.  The first step, and any step whose bed inputs, meshes or
 * parameters differ from the previous one, runs every bed eagerly (forked
 * from and joined to the batch's stream) and then captures the whole
 * ensemble -- binning, QCM, projection with device-driven CG loops, forces
 * and sources of all beds as parallel branches -- into one CUDA graph; later
 * identical steps replay it with a single launch.  Results equal those of
 * cfdem_coupling_step on each bed alone up to the order of the atomic
 * additions inside the fluid source and the PCM element volumes
 * (rounding); the void fraction and the forces are identical. */
typedef struct cfdem_batch *cfdem_batch_t;

/* Per-bed arguments of cfdem_batch_coupling_step: those of
 * cfdem_coupling_step (device pointers on the batch's device), then
 * optional host buffers (NULL = none) for a step that starts and ends in
 * host memory.  host_x and host_r are uploaded into x and r first;
 * host_u_p, host_u_nodal and host_p_nodal into u_p, u_nodal and p_nodal on
 * a second stream of the bed, while the void fraction and the projection
 * run (the forces wait for them); f and F_elem are downloaded into host_f
 * and host_F_elem at the end.  The device buffers are written although
 * declared const.  Host buffers must be page-locked (cudaHostAlloc or
 * registered) for the copies to overlap and for the step to be captured
 * into the batch's graph; they are part of the arguments a replay is keyed
 * on.  Sizes: x, u_p, f 3n; r n; u_nodal 3 n_nodes; p_nodal the pressure
 * nodes; F_elem 3 E doubles. */
typedef struct {
    int64_t n;
    const double *x, *r, *u_p, *u_nodal, *p_nodal;
    double *eps_nodal, *f, *f_drag, *F_elem, *F_q;
    const double *host_x, *host_r, *host_u_p, *host_u_nodal, *host_p_nodal;
    double *host_f, *host_F_elem;
} cfdem_bed_io;

/* Create a batch of n_beds (1 .. 4096) empty beds on `device`; `stream`
 * (a cudaStream_t, NULL = legacy default) orders the batch against the
 * caller's work. */
cfdem_status cfdem_batch_create(cfdem_batch_t *out, int device, void *stream, int n_beds);
/* Synchronise and release the batch, its graph and its bed contexts. */
cfdem_status cfdem_batch_destroy(cfdem_batch_t b);
/* The context of bed i, owned by the batch: give it a mesh and parameters
 * with cfdem_set_mesh / cfdem_set_params, read its statistics with
 * cfdem_get_stats after cfdem_batch_synchronize.  NULL if i is out of range.
 * A bed whose step cannot be captured (stage timers on, a mixed solve
 * without the fast-diagonalisation preconditioner, or host buffers that are
 * not page-locked) keeps the whole batch eager. */
cfdem_t cfdem_batch_bed(cfdem_batch_t b, int i);
/* 1 (default): capture and replay graphs; 0: always run the beds eagerly. */
cfdem_status cfdem_batch_set_graph(cfdem_batch_t b, int enable);
/* One coupling step of every bed; io[n_beds] (host array).  Returns without
 * synchronising; CFDEM_EINVAL for a bad argument, or the first failing
 * bed's status (cfdem_last_error of that bed tells why). */
cfdem_status cfdem_batch_coupling_step(cfdem_batch_t b, const cfdem_bed_io *io);
/* Wait for the batch; then as cfdem_synchronize on every bed.  Returns the
 * first bed's error (its index in *first_failed_bed, else -1), or CFDEM_OK. */
cfdem_status cfdem_batch_synchronize(cfdem_batch_t b, int *first_failed_bed);
/* 1 if the last step was a graph replay, 0 if it ran eagerly. */
int cfdem_batch_last_replayed(cfdem_batch_t b);
/* Text of the batch's last failure (empty if none); owned by the batch. */
const char *cfdem_batch_last_error(cfdem_batch_t b);

/* Wait for the context's stream and return the first device-side error of
 * the calls since the last synchronize (CFDEM_OUT_OF_DOMAIN,
 * CFDEM_NOT_CONVERGED) or CFDEM_OK. */
cfdem_status cfdem_synchronize(cfdem_t ctx);

/* Synchronize, then copy the counters into *out. */
cfdem_status cfdem_get_stats(cfdem_t ctx, cfdem_stats *out);

/* Largest element count accepted by cfdem_pcm_void_fraction_static. */
#define CFDEM_PCM_STATIC_MAX_ELEMS 524288

/* Particle-centroid void fraction that allocates nothing.  The paper has no
 * counterpart: this is a service to callers that cannot allocate device
 * memory -- solvers that hand all of the GPU's memory to their own pool, and
 * loops that must not take the device-wide synchronisation a cudaMalloc may
 * cause.
 * It needs no context: mesh as in cfdem_set_mesh (host arrays), particles
 * x_dev[n][3], r_dev[n] and the output eps_q_dev[E][Q] on the current device,
 * work ordered on `stream` (a cudaStream_t, NULL = legacy default).  The
 * result equals cfdem_void_fraction with scheme = 1 (eps_e = (V_e - sum of
 * V_p,i of the particles centred in e) / V_e on every Gauss point of e).
 *   - The per-element scratch is one fixed device array of
 *     CFDEM_PCM_STATIC_MAX_ELEMS doubles (4 MiB) compiled into the library
 *     and kept by every GPU that loads it until the process exits; meshes
 *     with more elements return CFDEM_EINVAL.
 *   - The first call on a device looks the array's address up (no
 *     allocation); make that first call before any stream capture.
 *   - All calls share the array: each call clears it on its stream before
 *     use, but calls that overlap on the GPU (on different streams, or from
 *     several threads) race on it and must be serialised by the caller.
 *   - Particles outside the mesh are left out and not reported.
 * Returns CFDEM_EINVAL on bad arguments or too many elements, CFDEM_ECUDA if
 * a CUDA call fails, else CFDEM_OK without synchronising. */
cfdem_status cfdem_pcm_void_fraction_static(const double origin[3], const double extent[3],
                                            const int n_el[3], int degree, int64_t n,
                                            const double *x_dev, const double *r_dev,
                                            double *eps_q_dev, void *stream);

/* Turn the per-stage CUDA-event timers on (1) or off (0) and reset them and
 * the launch counter.  Synchronizes the stream.  Timers record an event pair
 * per stage and per operator launch; they do not change results. */
cfdem_status cfdem_set_timing(cfdem_t ctx, int enable);

/* Text of the last error on this context ("" if none).  Owned by ctx. */
const char *cfdem_last_error(cfdem_t ctx);

/* Library version string. */
const char *cfdem_version(void);

/* --------------------------------------------------- mapped (curved) meshes */

/* Particle location on a mapped Q_k hex mesh.  The paper's beds sit in
 * curved meshes (a subdivided cylinder, Secs. 3.1 and 3.2; a gmsh mesh,
 * Sec. 3.4), and particles are located on the fluid mesh itself (Sec. 2.3).
 * Element e maps the reference cube [0,1]^3 by its Q_k nodes (GLL points):
 * X_e(xi) = sum_{a,b,c} P[conn[e][a + (k+1)(b + (k+1) c)]] l_a(xi_0) l_b(xi_1)
 * l_c(xi_2); x lies in e when X_e(xi) = x for a xi in the cube.  The box
 * mesh entry points above are the special case of an axis-aligned box. */
typedef struct cfdem_mapped *cfdem_mapped_t;

/* Copy a mapped mesh to `device`: degree 1..3, n_elem elements, conn[n_elem]
 * [(degree+1)^3] node indices (host, a fastest; right-handed reference axes
 * with positive Jacobian), nodes[n_nodes][3] coordinates (host).  Each
 * element's candidate box is its nodes' box widened on every side by
 * `margin` (in [0, 1]) times its largest edge (0.1 covers the bulge of
 * curved Q2/Q3 faces beyond their nodes).  CFDEM_EINVAL on a bad argument
 * (an index outside [0, n_nodes), a non-finite coordinate), CFDEM_ECUDA /
 * CFDEM_ENOMEM on device failures.  Host arrays are not kept. */
cfdem_status cfdem_mapped_create(cfdem_mapped_t *out, int device, int degree, int64_t n_elem,
                                 const int32_t *conn, int64_t n_nodes, const double *nodes,
                                 double margin);
cfdem_status cfdem_mapped_destroy(cfdem_mapped_t mesh);

/* Element elem_dev[n] and reference coordinates xi_dev[n][3] (may be NULL)
 * of each particle x_dev[n][3] (device arrays): the elements whose candidate
 * box contains the particle are tried in ascending index by Newton's method
 * on X_e(xi) = x from the cube's centre (FP64, at most 50 steps, converged at
 * a step of at most 1e-13, abandoned once xi leaves [-3, 4]^3 or the
 * Jacobian is singular); the first whose xi lies in [-1e-10, 1 + 1e-10]^3
 * is the element, xi clamped to [0,1]^3.  A particle in no element gets
 * elem = -1 and xi = 0 (not an error).  Stream ordered on `stream` (a
 * cudaStream_t, NULL = legacy default). */
cfdem_status cfdem_mapped_locate(cfdem_mapped_t mesh, int64_t n, const double *x_dev,
                                 int32_t *elem_dev, double *xi_dev, void *stream);

/* out_dev[n][ncomp] = the Q_k interpolant of the nodal field field_dev
 * [n_nodes][ncomp] at (elem_dev[i], xi_dev[i]) (0 where elem < 0), e.g. the
 * fluid velocity at the particles located by cfdem_mapped_locate; ncomp in
 * 1..64.  Device arrays, stream ordered. */
cfdem_status cfdem_mapped_interpolate(cfdem_mapped_t mesh, int64_t n, const int32_t *elem_dev,
                                      const double *xi_dev, int ncomp, const double *field_dev,
                                      double *out_dev, void *stream);

/* ------------------------------------------------------------------ DEM */

/* The particle side of the coupling (Sec. 2.2): Newton's laws for
 * translation and rotation, Eqs. (newton_law) and (angular_momentum),
 *   m dv/dt = sum_j f_ij + sum_w f_wi + m g + f_fp,  I dw/dt = sum_j (M^t + M^r),
 * I = 2/5 m r^2, with soft-sphere contacts of the non-linear visco-elastic
 * model of Table (viscoelastic): k_n = 4/3 Y_e sqrt(R_e d_n), eta_n =
 * -2 sqrt(5/6) beta sqrt(S_n m_e), k_t = 8 G_e sqrt(R_e d_n), eta_t =
 * -2 sqrt(5/6) beta sqrt(S_t m_e), beta = ln e / sqrt(ln^2 e + pi^2), the
 * effective mass, radius and moduli of the table, f^n = -k_n d_n n -
 * eta_n v_rn, f^t = -k_t d_t - eta_t v_rt; Velocity Verlet integration
 * (Sec. 2.2), sub-cycled with the fluid force f_fp held (the DEM frequency
 * f_coupling of Sec. 2.3).  Readings: the tangential displacement d_t is
 * kept per contact, turned onto the current tangent plane and advanced by
 * v_rt dt; the Coulomb limit mu_s |f^n| caps f^t (and resets d_t to match);
 * rolling resistance is the constant-torque form -mu_r R_e |f^n| w_rel /
 * |w_rel|; the six faces of the box [lo, hi] are walls of infinite mass and
 * radius; forces at step n+1 use positions x(n+1) and half-step velocities. */
typedef struct cfdem_dem *cfdem_dem_t;

typedef struct {
    double rho_p;                 /* particle density [kg/m^3] */
    double youngs, poisson;       /* particle Young's modulus [Pa], Poisson ratio */
    double restitution;           /* particle-particle coefficient of restitution e, (0, 1] */
    double friction;              /* sliding friction mu_s */
    double rolling_friction;      /* rolling friction mu_r */
    double wall_youngs, wall_poisson, wall_restitution, wall_friction, wall_rolling_friction;
    double g[3];                  /* gravity [m/s^2] */
    double lo[3], hi[3];          /* the walls: faces of the box [lo, hi] */
    double max_radius;            /* the largest particle radius (cell size 2 max_radius) */
    int capacity;                 /* contacts kept per particle, 1..64 (default 24) */
    int precision;                /* 0 = FP64 (default); 1 = mixed: FP64 positions,
                                     velocities, contact test and the difference of
                                     squares behind each overlap; FP32 contact forces
                                     and carried tangential displacements */
} cfdem_dem_params;

/* Glass-like defaults (rho 2500, Y 1e7, nu 0.3, e 0.9, mu_s 0.3, mu_r 0,
 * walls alike), g = (0, 0, -9.81), capacity 24; the box and max_radius
 * are left 0 and must be set. */
void cfdem_dem_params_default(cfdem_dem_params *p);

/* A DEM state on CUDA device `device`, work ordered on `stream`. */
cfdem_status cfdem_dem_create(cfdem_dem_t *out, int device, void *stream);
cfdem_status cfdem_dem_destroy(cfdem_dem_t dem);

/* Set (or change) the parameters; CFDEM_EINVAL for a bad value.  The
 * carried accelerations are recomputed at the next step; a change of
 * capacity or precision also forgets the contact history. */
cfdem_status cfdem_dem_set_params(cfdem_dem_t dem, const cfdem_dem_params *p);

/* Forget the contact history and the carried accelerations. */
cfdem_status cfdem_dem_reset(cfdem_dem_t dem);

/* nsub Velocity Verlet sub-steps of length dt, in place: x_dev, v_dev, w_dev
 * [n][3] (positions, velocities, angular velocities, device, FP64), radii
 * r_dev[n], fluid force f_ext_dev[n][3] held over the sub-steps (NULL =
 * none).  The contact history (tangential displacements per particle pair
 * and per wall) and the last accelerations carry over to the next call
 * while n stays the same and particle i stays particle i; a different n
 * starts afresh.  Stream ordered; a particle with more than `capacity`
 * contacts (its extra contacts are dropped) or a radius above max_radius
 * is reported by the next cfdem_dem_synchronize. */
cfdem_status cfdem_dem_step(cfdem_dem_t dem, int64_t n, double *x_dev, double *v_dev,
                            double *w_dev, const double *r_dev, const double *f_ext_dev,
                            double dt, int nsub);

/* Wait for the stream; CFDEM_ECAPACITY or CFDEM_EINVAL (radius above
 * max_radius) if a step since the last call met one (the flag is cleared). */
cfdem_status cfdem_dem_synchronize(cfdem_dem_t dem);

/* Text of the last error on this DEM state. */
const char *cfdem_dem_last_error(cfdem_dem_t dem);

#ifdef __cplusplus
}
#endif

#endif /* CFDEM_H */
