/*
 * yk.h - C ABI of a GB300 (sm_103a) solver for the exterior screened-Laplace
 * (Yukawa) Dirichlet problem on the boundaries of rigid planar Janus
 * particles, and the hydrophobic forces and torques it induces
 * (Fu, Ryham, Kloeckner, Wala, Jiang, Young, arXiv 1810.04131).
 *
 * Problem (Section 1, Eq. SL): -rho^2 Lap u + u = 0 in the water region,
 * u = f on the particle boundaries, u -> 0 at infinity. The solution is
 * represented as a double-layer potential u = D[sigma] (Eq. intrep) with
 * kernel dG/dnu_y, G = K0(|x-y|/rho)/(2 pi) (Eqs. Gfunc, double-layer-def);
 * sigma solves the second-kind equation 1/2 sigma + D sigma = f (Eq. bie).
 * Discretisation: composite Gauss-Legendre panels (Nystrom) with one-sided
 * exterior QBX on the target's own panel and its neighbours (Section 5).
 * Forces and torques are the boundary integrals of the hydrophobic stress
 * (Eqs. stress, force_torque, scalar-torque).
 *
 * Conventions for every call:
 *   - Return value: YK_OK (0) or a negative YK_ERR_* code; yk_strerror()
 *     gives a message. No call aborts, traps or exits.
 *   - Array arguments are caller-owned. Each may be a host pointer or a
 *     CUDA device pointer (decided per pointer by cudaPointerGetAttributes);
 *     host arrays are staged through library-owned device buffers, so a call
 *     with host arrays includes the host<->device copies.
 *   - Arrays are dense, C-contiguous, FP64 unless stated. Node arrays have
 *     length N = n_particles * n_panels * n_gl, ordered particle-major, then
 *     panel, then Gauss-Legendre node. Point arrays are interleaved (x, y).
 *   - All work is enqueued on the context's CUDA stream; calls that return
 *     host-visible results synchronise that stream before returning.
 *   - Opaque handles are owned by the library and released by yk_destroy*.
 *   - A context and the geometries made from it are not thread-safe: use
 *     one host thread per context.
 */
#ifndef YK_H
#define YK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define YK_OK                  0
#define YK_ERR_ARG            -1  /* bad argument (null, size, range)          */
#define YK_ERR_BAD_GEOMETRY   -2  /* particles overlap or touch               */
#define YK_ERR_NO_MEMORY      -3  /* device or host allocation failed         */
#define YK_ERR_NOT_CONVERGED  -4  /* solver stopped above tolerance; outputs
                                     still written with the achieved residual */
#define YK_ERR_TIMEOUT        -5  /* a bounded device wait gave up            */
#define YK_ERR_CUDA           -6  /* a CUDA runtime call failed               */
#define YK_ERR_NOT_FOUND      -7  /* unknown request id                       */
#define YK_ERR_BUSY           -8  /* serving queue full                        */
#define YK_ERR_TOO_LARGE      -9  /* request exceeds a fixed, preallocated limit */

/* ---- enumerations --------------------------------------------------------- */
#define YK_SHAPE_DISK     0
#define YK_SHAPE_ELLIPSE  1

#define YK_FP64   0   /* every step in FP64                                   */
#define YK_MIXED  1   /* FP32 far-field evaluation with FP64 accumulation inside
                         an FP64 iterative-refinement outer solve              */

#define YK_REP_DOUBLE_LAYER 0 /* u = D[sigma] (Eq. intrep), equation Eq. bie    */
#define YK_REP_COMBINED     1 /* u = D[sigma] + bw_eta S[sigma] (the combined
                                 representation of the remark on Eq. bwform,
                                 with a real coupling: S of Eq.
                                 single-layer-def); the equation becomes
                                 1/2 sigma + D sigma + bw_eta S sigma = f,
                                 whose weak modes at large rho are lifted.
                                 YK_FP64 precision, dense or cut-off far
                                 field; yk_eval_potential_near is not
                                 available with it                          */

#define YK_PRECOND_NONE   0  /* plain GMRES                                   */
#define YK_PRECOND_BLOCK  1  /* right preconditioning by the inverse of each
                                particle's self-interaction block (the same
                                block for all particles of one shape)        */

#define YK_COARSE_NONE    0  /* the inner GMRES sees block Jacobi alone       */
#define YK_COARSE_MODES   1  /* YK_MIXED with YK_PRECOND_BLOCK: the inner
                                (FP32) GMRES is deflated by a coarse space of
                                three density modes per particle (1, cos and
                                sin of the polar angle about its centre): the
                                coupling of every particle's lowest modes to
                                its neighbours is stored (B Z, per target
                                particle, for source particles whose coupling
                                exceeds 1e-9 x max|sigma|) and Z^T B Z
                                (3 np square) is inverted once per
                                configuration. Used for 2..2048 particles
                                without near-contact panels and with at most
                                2 GiB of stored couplings; otherwise the
                                solve runs with block Jacobi alone          */

#define YK_FARFIELD_DENSE  0  /* every far source pair evaluated              */
#define YK_FARFIELD_CUTOFF 1  /* source particles whose whole contribution is
                                 bounded below cutoff_tol * max|sigma| are
                                 left out (cut-off localisation, Section 3.3);
                                 the K1 kernel decays like exp(-r/rho)        */
#define YK_FARFIELD_FMM    2  /* YK_MIXED: the inner (FP32) operator's far
                                 field by a uniform-quadtree fast multipole
                                 method (multipole/local expansions of order
                                 fmm_order by Graf's addition theorem, the
                                 Yukawa form of Eq. graf-addition); particles
                                 in leaves at most two boxes apart interact
                                 directly. The refinement residuals, the
                                 normal derivative and YK_FP64 use the
                                 YK_FARFIELD_CUTOFF operator, so results keep
                                 the accuracy of that operator               */

/* Dirichlet data generators; theta is the polar angle of x - a_i measured
 * from the director d_i = (cos phi_i, sin phi_i) (Section 2.1).           */
#define YK_LABEL_TANH    0   /* f = (1 + tanh(param cos theta)) / 2            */
#define YK_LABEL_SINP    1   /* f = 1 - sin^param theta, Eq. JanusBC           */
#define YK_LABEL_COS     2   /* f = (1 + cos theta) / 2 (Eq. true_soln data)   */
#define YK_LABEL_CUSTOM  3   /* f supplied by the caller                       */

/* serving request status */
/* Stokes operators (yk_stokes_apply; Section 3). */
#define YK_STOKES_TRACTION  0 /* (1/2 I + K*) sigma: traction of S[sigma] on the
                                 inside of each boundary (Eq. stokesjump)     */
#define YK_STOKES_COMPLETED 1 /* (1/2 I + K* + W) sigma: the operator of the
                                 mobility equation (W: rigid-motion projector) */
#define YK_STOKES_VELOCITY  2 /* S[sigma] on the boundary: the stokeslet single
                                 layer of Eq. mobilityu                      */

#define YK_REQ_QUEUED   0
#define YK_REQ_RUNNING  1
#define YK_REQ_DONE     2
#define YK_REQ_FAILED   3

/* ---- data types ----------------------------------------------------------- */
typedef struct yk_ctx yk_ctx;
typedef struct yk_geom yk_geom;

/* One rigid particle (Section 2.1): boundary x(t) = (cx, cy) +
 * R(phi) (A cos t, B sin t), t in [0, 2 pi); A is the semi-axis along the
 * director. A disk has A = B = radius.                                      */
typedef struct {
    int32_t shape;      /* YK_SHAPE_DISK or YK_SHAPE_ELLIPSE                  */
    int32_t pad_;
    double cx, cy;      /* centre a_i                                        */
    double phi;         /* orientation theta_i of the director d_i           */
    double A, B;        /* semi-axes                                         */
} yk_particle;

/* Numerical parameters. yk_default_params() fills the defaults given here. */
typedef struct {
    double rho;            /* screening length (Eq. SL); default 1            */
    double gamma;          /* interfacial tension (Eq. main); default 1       */
    int32_t n_panels;      /* panels per particle; default 16                 */
    int32_t n_gl;          /* Gauss-Legendre nodes per panel, 2..32; default 16 */
    int32_t qbx_order;     /* QBX order p, terms |n| <= p, 1..24; default 10  */
    int32_t oversample;    /* QBX sub-panels per near panel; default 8        */
    double qbx_r_factor;   /* expansion radius r = factor * panel arclength; 1/8 */
    int32_t near_width;    /* near panels on each side of the target's; default 1 */
    int32_t gmres_restart; /* Krylov basis size m; default 100                */
    int32_t max_iter;      /* total GMRES iterations (all restarts); default 300 */
    int32_t precision;     /* YK_FP64 or YK_MIXED; default YK_MIXED            */
    double gmres_tol;      /* relative residual ||f - A sigma|| / ||f||; default
                              1e-12. The forces and torques amplify the density
                              error (about 25x for ellipses at rho = 4), so a
                              residual of 1e-10 leaves them only within a few
                              1e-9 of the exact discrete solution; at 1e-12 the
                              density, forces and torques are within 1e-11    */
    double inner_tol;      /* YK_MIXED: inner (FP32) GMRES tolerance; 1e-6     */
    int32_t max_refine;    /* YK_MIXED: refinement steps; default 8            */
    int32_t farfield;      /* YK_FARFIELD_DENSE, _CUTOFF or _FMM; default DENSE */
    double split_tol;      /* YK_MIXED refinement residual: a source particle is
                              evaluated in FP32 only where its FP32 error bound
                              is below split_tol * max|sigma|; default 1e-14.
                              The bounds decay like exp(-gap/rho), so their sum
                              over all FP32 particles is a small multiple of
                              one bound (about 2x at 4% area fraction)       */
    double grad_split_tol; /* the same bound for the normal derivative that
                              feeds the forces (YK_MIXED); default 1e-13       */
    int32_t precond;       /* YK_PRECOND_NONE or YK_PRECOND_BLOCK (needs
                              n_panels * n_gl <= 1024); default BLOCK        */
    int32_t pad_;
    double cutoff_tol;     /* YK_FARFIELD_CUTOFF: a source particle is dropped
                              for a target particle when its contribution
                              (value or normal derivative) is bounded below
                              cutoff_tol * max|sigma|; default 1e-15 (also
                              bounds the reach of YK_FARFIELD_FMM)           */
    int32_t fmm_order;     /* YK_FARFIELD_FMM: expansion order p, terms
                              |n| <= p, 2..30; default 12                    */
    int32_t pad2_;
    double fmm_leaf;       /* YK_FARFIELD_FMM: leaf box side; 0 (default)
                              chooses it by timing the admissible leaf sizes
                              on the first FMM operator application          */
    int32_t representation;/* YK_REP_DOUBLE_LAYER (default) or YK_REP_COMBINED */
    int32_t pad3_;
    double bw_eta;         /* YK_REP_COMBINED: coupling eta > 0 of the single
                              layer; default 0.25 (on six ellipses, plain GMRES
                              to 1e-12 takes 25-26 iterations at rho = 4-16
                              against 34-45 for the double layer alone)      */
    double viscosity;      /* Stokes mobility: fluid viscosity mu of Eq. stokes;
                              default 1 (the non-dimensional mu = 1 of the
                              paper's time scale [T] = mu a / gamma)          */
    int32_t coarse;        /* YK_COARSE_NONE or YK_COARSE_MODES; default MODES */
    int32_t pad4_;
} yk_params;

/* Constant-drag dynamics (Eq. euler) with the excluded-volume repulsion of
 * Eq. repul. yk_default_dynamics() fills the defaults given here.           */
typedef struct {
    double dt;             /* time step Delta t; default 0.1                   */
    double xi_x;           /* translational drag xi_x; default 4 pi (Section
                              S2: 4 pi mu a with mu = a = 1)                  */
    double xi_theta;       /* rotational drag xi_theta; default 4 pi          */
    double c0;             /* repulsion strength c0 of Eq. repul; default 0.01 */
    int32_t q;             /* repulsion order q; default 3 (two dimensions)    */
    int32_t label_kind;    /* Dirichlet data each step: YK_LABEL_TANH, _SINP or
                              _COS (the label turns with its particle);
                              default YK_LABEL_TANH                          */
    double label_param;    /* its parameter; default 10                      */
    int32_t warm_start;    /* 1 (default): the previous step's density is the
                              initial guess of the next solve                 */
    int32_t mobility;      /* 0 (default): constant drag, Eq. euler with xi_x,
                              xi_theta; 1: the particle velocities from the
                              Stokes mobility problem (yk_mobility), Eq.
                              mob_vec by forward Euler                        */
} yk_dynamics;

/* Solve statistics (all host memory). */
typedef struct {
    int32_t iterations;      /* GMRES iterations (inner ones for YK_MIXED)    */
    int32_t refinements;     /* outer refinement steps (YK_MIXED) or 0        */
    double rel_residual;     /* final ||f - A sigma|| / ||f|| in FP64         */
    int32_t matvecs_fp64;    /* FP64-accurate operator applications           */
    int32_t matvecs_fp32;    /* FP32 far-field operator applications          */
    int32_t coarse_dim;      /* columns of the coarse space that deflated the
                                inner GMRES (3 per particle, YK_COARSE_MODES),
                                0 when the solve ran without one              */
} yk_solve_info;

/* ---- context -------------------------------------------------------------- */

/* Fill *p with the defaults documented in yk_params. Never fails for p != NULL. */
int yk_default_params(yk_params* p);

/* Create a context on CUDA device `device`, enqueuing all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream). The
 * stream is borrowed, not owned. Errors: YK_ERR_ARG, YK_ERR_CUDA.        */
int yk_create(yk_ctx** ctx, int device, void* cuda_stream);
/* Destroy a context, and with it every geometry made from it that is still
 * alive and every pending serving request; their handles become invalid. */
int yk_destroy(yk_ctx* ctx);

/* ---- geometry (Section 2.1; Section 5: discretisation and QBX set-up) ----- */

/* Discretise n_particles particles with parameters *prm: nodes, normals,
 * weights (composite Gauss-Legendre panels), per-panel arclength, the QBX
 * near-correction rows (value and normal derivative; one block per distinct
 * particle shape, since the rows of a rigid body do not depend on its
 * position or orientation), and the solver workspace. The particle array
 * is host memory and is copied.
 * Errors: YK_ERR_ARG (sizes/parameters out of range), YK_ERR_BAD_GEOMETRY
 * (two particles' bounding circles overlap: the disks-and-ellipses
 * configurations used here keep a positive surface gap), YK_ERR_NO_MEMORY. */
int yk_create_geometry(yk_ctx* ctx, const yk_particle* particles, int n_particles,
                       const yk_params* prm, yk_geom** out);
int yk_destroy_geometry(yk_geom* g);

/* Move the particles of an existing geometry (Algorithm 1, position and
 * orientation update followed by re-discretisation): same count, same
 * shapes and semi-axes, new centres and orientations (host array). Nodes,
 * normals and weights are recomputed; the QBX near rows are kept, because
 * a rigid particle's rows do not depend on its position or orientation.
 * Errors: YK_ERR_ARG (count or shapes differ, non-finite values). The
 * overlap check of yk_create_geometry is not repeated.                   */
int yk_update_geometry(yk_geom* g, const yk_particle* particles, int n_particles);

/* N = n_particles * n_panels * n_gl (host int64). */
int yk_num_nodes(const yk_geom* g, int64_t* n);

/* Copy node positions xy (N x 2), unit normals nrm (N x 2, out of the
 * particle), and weights w (N). Any output may be NULL.                   */
int yk_nodes(const yk_geom* g, double* xy, double* nrm, double* w);

/* Dirichlet data f at the nodes (Eq. JanusBC and variants): kind is one of
 * YK_LABEL_*; param is the tanh steepness or the sin exponent. For
 * YK_LABEL_CUSTOM f_custom (N) is copied to f_out. f_out has length N.    */
int yk_label(yk_geom* g, int kind, double param, const double* f_custom, double* f_out);

/* y = (1/2 I + D) sigma (Eq. bie), both of length N. precision YK_FP64:
 * every pair in FP64. YK_MIXED: FP32 far field with FP64 accumulation
 * (the inner operator of the mixed solver, accurate to about 1e-6).       */
int yk_matvec(yk_geom* g, const double* sigma, double* y, int precision);

/* Normal derivative u_nu = nu . grad D[sigma] on the boundary, exterior
 * limit (Algorithm 1, step computing grad u), length N. precision YK_FP64
 * or YK_MIXED (precision-split: FP64 where FP32 would exceed split_tol). */
int yk_normal_derivative(yk_geom* g, const double* sigma, double* u_nu, int precision);

/* Solve 1/2 sigma + D sigma = f (Eq. bie) by restarted GMRES (YK_FP64) or
 * FP64 iterative refinement over FP32-operator GMRES (YK_MIXED), as set in
 * the geometry's parameters: right block preconditioner (precond), and for
 * YK_MIXED the inner GMRES deflated by the coarse space (coarse). The
 * stopping test is on the FP64 residual ||f - A sigma|| / ||f|| of the
 * plain operator, whatever preconditions the inner solve. sigma0 (N,
 * nullable) is an initial guess (warm start); sigma (N) receives the
 * solution; info (host, nullable) receives statistics. Returns
 * YK_ERR_NOT_CONVERGED if the tolerance was not reached (sigma then holds
 * the last iterate). The first preconditioned solve on a geometry
 * allocates the preconditioned Krylov basis (gmres_restart x N doubles) and
 * the coarse space; a solve after the particles moved rebuilds the latter. */
int yk_solve(yk_geom* g, const double* f, double* sigma, const double* sigma0,
             yk_solve_info* info);

/* Solve 1/2 sigma + D sigma = f (Eq. bie) for count independent
 * configurations at once, each to its own parameters and tolerance, with the
 * results of count separate yk_solve calls (from a zero initial guess) up to
 * the solver tolerance. The inner FP32 GMRES of every mixed-precision,
 * dense-far-field system with self blocks and the block preconditioner (and
 * no near-contact pairs) advances in lock step with the others: each step is
 * one kernel launch per stage for all of them. Other systems are solved one
 * after another as by yk_solve.
 *   - geoms (count): distinct geometries of one context;
 *   - f, sigma (count arrays of N_s each, per pointer host or device);
 *   - info (count, host, nullable): the statistics of each system.
 * Returns YK_ERR_NOT_CONVERGED if some system stopped above its tolerance
 * (its sigma holds the last iterate), another error code if one failed. */
int yk_solve_batch(yk_geom* const* geoms, int count, const double* const* f,
                   double* const* sigma, yk_solve_info* info);

/* Forces F (n_particles x 2) and scalar torques tau (n_particles) about the
 * particle centres (Eqs. force_torque, stress, scalar-torque) from the
 * density sigma and the data f, using u_nu from yk_normal_derivative (in
 * the geometry's precision mode) and u_tau = df/ds by per-panel spectral
 * differentiation. net (3, nullable) receives sum F_x, sum F_y and
 * sum tau0 (torque about the origin), which vanish by Eq. net.            */
int yk_forces_torques(yk_geom* g, const double* sigma, const double* f,
                      double* F, double* tau, double* net);

/* Energy of Eq. main, Phi = gamma min I[u] with I[u] = int rho |grad u|^2 +
 * u^2/rho over the water, in its boundary form (Green's first identity with
 * Delta u = u / rho^2): Phi = -gamma rho sum_i int_{Sigma_i} f du/dnu ds, with
 * u_nu from sigma as in yk_forces_torques (the solved density of f).
 *   - phi (n_particles, nullable): the per-particle parts
 *     -gamma rho int_{Sigma_i} f u_nu ds;
 *   - phi_total (1, nullable): Phi; at least one of the two must be given.
 * Its centered differences in a particle's position and angle are minus the
 * force and torque of yk_forces_torques (Section 7.1).                     */
int yk_energy(yk_geom* g, const double* sigma, const double* f, double* phi,
              double* phi_total);

/* Excluded-volume repulsion at the geometry's current positions: an ellipse
 * is three circles of radius B at a_i + k (A - B) d_i, k in {-1, 0, 1}, a disk
 * one circle (Section S1); every pair of circles of different particles
 * repels by Eq. repul with c0 / (n_i n_j) (n circles per particle), so that
 * circles recover Eq. repul exactly. F (2 n_particles), tau (n_particles,
 * torque about a_i from the circles' lever arms) and phi (n_particles, half
 * of each pair's potential c / gap^q) may each be NULL. YK_ERR_BAD_GEOMETRY
 * if two circles overlap.                                                   */
int yk_repulsion(yk_geom* g, double c0, int q, double* F, double* tau, double* phi);

int yk_default_dynamics(yk_dynamics* d);

/* Algorithm 1: n_steps forward-Euler steps, each one Dirichlet label, GMRES
 * (yk_solve, warm-started from the previous step's density when
 * d->warm_start), the hydrophobic force and torque (yk_forces_torques), the
 * repulsion (yk_repulsion), then with constant drag (d->mobility = 0, Eq.
 * euler)
 *   a_i += dt (F_i + F_rep_i) / xi_x,  theta_i += dt (tau_i + tau_rep_i) / xi_theta,
 * or with the Stokes mobility (d->mobility = 1, Eq. mob_vec)
 *   (v, omega) = yk_mobility(F + F_rep, tau + tau_rep),
 *   a_i += dt v_i,  theta_i += dt omega_i,
 * and the re-discretisation at the new positions (yk_update_geometry).
 *   - particles (n_particles, nullable): the positions after the last step;
 *   - energy (n_steps, nullable): Phi of Eq. main plus the repulsion
 *     potential at the configuration each step starts from;
 *   - info (n_steps, nullable): the solve statistics of each step.
 * Stops at the first failing step (YK_ERR_NOT_CONVERGED, or
 * YK_ERR_BAD_GEOMETRY when particles overlap) with the particles where that
 * step found them.                                                         */
int yk_step(yk_geom* g, const yk_dynamics* d, int n_steps, yk_particle* particles,
            double* energy, yk_solve_info* info);

/* u = D[sigma] (Eq. intrep) at nt off-surface targets (nt x 2) by plain
 * quadrature, FP64. Targets must lie in the water at least about one panel
 * length from every boundary for full accuracy. u has length nt.          */
int yk_eval_potential(yk_geom* g, const double* sigma, const double* targets,
                      int64_t nt, double* u);

/* u = D[sigma] (Eq. intrep) at nt targets (nt x 2) anywhere in the water,
 * including targets arbitrarily close to a boundary (the paper's Table 1
 * samples such targets on a grid), FP64. Panels next to a target (within one
 * largest panel arclength of its closest boundary point, found by Newton's
 * method on the curve parameter) are evaluated by QBX (Section 5) about a
 * centre on the normal through that closest point (target within twice the
 * expansion radius of the boundary) or by quadrature on their oversampled
 * nodes (farther); all other panels by plain quadrature. A target inside a
 * particle gets NaN. YK_ERR_TOO_LARGE when a target lies in the near zone of
 * more than four particles.                                                 */
int yk_eval_potential_near(yk_geom* g, const double* sigma, const double* targets,
                           int64_t nt, double* u);

/* Allocation-free variant of yk_eval_potential. The paper has no
 * counterpart. It is for callers that must not allocate device memory at the
 * point where they evaluate the potential: a real-time loop that cannot
 * block in the allocator (an allocation may synchronise the device and has
 * no latency bound), or an application that reserved the GPU's memory up
 * front and hands libraries a fixed budget. It computes the same
 * u = D[sigma] at nt off-surface targets as yk_eval_potential, but keeps its
 * partial sums in a fixed 8 MiB device array inside the library (one per
 * GPU that loads the library, held until the process exits) and allocates
 * nothing.
 *   - sigma (N), targets (nt x 2) and u (nt) must be device memory of the
 *     context's device (YK_ERR_ARG otherwise: staging host arrays would
 *     allocate).
 *   - nt <= 1,048,576 (2^20); larger requests return YK_ERR_TOO_LARGE.
 *   - The first call on each device looks up the array's device address and
 *     keeps it for the life of the process; make that first call before any
 *     stream capture begins. A device reset (cudaDeviceReset) invalidates the
 *     kept address: do not call this entry point after one.
 *   - All calls share the array, which keeps the last call's contents (every
 *     partial sum a call reads, it wrote first). Calls whose kernels overlap
 *     on the GPU (two streams, or two contexts on one device) race on it:
 *     order them.
 *   - The call enqueues its work on the context's stream and returns without
 *     synchronising it.                                                      */
int yk_eval_potential_noalloc(yk_geom* g, const double* sigma, const double* targets,
                              int64_t nt, double* u);

/* Convenience: label + solve + forces for one configuration. */
int yk_solve_forces(yk_geom* g, const double* f, double* sigma, double* F,
                    double* tau, yk_solve_info* info);

/* ---- serving (continuous batching of independent configurations) --------- */

/* Queue one configuration (particles copied from host memory) to be solved
 * with the tanh/sin/cos label kind and parameter given, in parameters *prm.
 * The request is admitted when device memory allows, batched with the
 * others in flight, and its results are kept until yk_poll collects them.
 * Errors: YK_ERR_ARG, YK_ERR_BUSY (queue full).                           */
int yk_submit(yk_ctx* ctx, const yk_particle* particles, int n_particles,
              const yk_params* prm, int label_kind, double label_param,
              uint64_t* request_id);

/* Advance the serving loop and report request `id`. status receives a
 * YK_REQ_* value. When DONE, the outputs (host arrays, each nullable) are
 * written: sigma (N), F (2 n_particles), tau (n_particles), info, and
 * latency_ms (submit to completion); the request is then released.
 * Errors: YK_ERR_NOT_FOUND.                                                */
int yk_poll(yk_ctx* ctx, uint64_t id, int* status, double* sigma, double* F,
            double* tau, yk_solve_info* info, double* latency_ms);

/* Run the serving loop until every queued request is done (or a request
 * failed). Returns the first error met, or YK_OK; YK_ERR_TIMEOUT when no
 * request has completed for five minutes.                                  */
int yk_drain(yk_ctx* ctx);

/* Stokes boundary operators of the mobility problem (Section 3), on a
 * density sigma of 2 N values stored node by node (x and y component of node
 * 0, then node 1, ...), with nu the normal out of each particle:
 *   YK_STOKES_TRACTION:  out = 1/2 sigma + K* sigma, the traction of the
 *     stokeslet single layer u = S[sigma] on the inside of each boundary,
 *     K* sigma(x) = sum_y w_y T(x - y, nu(x)) sigma(y) with the stresslet
 *     T(r, n) = -(1/pi) r r^T (r . n) / |r|^4 (Eq. stokesjump with the target
 *     normal; the curvature limit -(kappa/(2 pi)) tau tau^T on the diagonal);
 *   YK_STOKES_COMPLETED: out = that plus W sigma, W the orthogonal projector
 *     on each boundary (weights w) onto the rigid motions (1, 0), (0, 1),
 *     (x - a_i)^perp;
 *   YK_STOKES_VELOCITY:  out = S[sigma] at the boundary nodes, the stokeslet
 *     G = (1/(4 pi mu)) (-log r I + r r^T / r^2) integrated with the log's
 *     singularity by product integration on each node's panel and its two
 *     neighbours (needs n_panels >= 3).
 * precision: YK_FP64, or YK_MIXED for the FP32 far field (YK_STOKES_COMPLETED
 * only; the others are always FP64). sigma, out: host or device, 2 N.
 * Needs n_panels >= 3 and n_panels * n_gl <= 512 (YK_ERR_ARG otherwise) and
 * at most 16384 particles (the particle-pair lists hold every pair;
 * YK_ERR_TOO_LARGE beyond).                                                 */
int yk_stokes_apply(yk_geom* g, int op, const double* sigma, double* out, int precision);

/* The Stokes mobility problem (Section 3: Eqs. stokes, mobility_bc,
 * stokesjump, mobilityu) of the geometry's particles under forces F
 * (2 n_particles) and torques tau (n_particles, about each centre a_i): the
 * density sigma = sigma_inc + mu, sigma_inc = F_i / |dP_i| + tau_i
 * (x - a_i)^perp / J_i (J_i = int |x - a_i|^2 ds) carrying the loads, mu from
 *   (1/2 I + K* + W) mu = -(1/2 I + K*) sigma_inc
 * (zero interior traction, so S[sigma] moves every boundary rigidly; mu
 * carries no force or torque), by GMRES (FP64) or mixed-precision GMRES with
 * iterative refinement (YK_MIXED: FP32 far field in the inner solves) to
 * gmres_tol; then the velocities of Eq. mobilityu,
 *   v_i = int_{dP_i} S[sigma] ds / |dP_i|,
 *   omega_i = int_{dP_i} (x - a_i) x S[sigma] ds / J_i.
 * Outputs v (2 n_particles), omega (n_particles), sigma (2 N, nullable),
 * info (nullable): host or device. Errors as yk_stokes_apply; outputs are
 * written with YK_ERR_NOT_CONVERGED too.                                    */
int yk_mobility(yk_geom* g, const double* F, const double* tau, double* v, double* omega,
                double* sigma, yk_solve_info* info);

/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts), for accounting in benchmarks. Library-specific; the
 * paper has no counterpart.                                               */
int yk_kernel_launches(uint64_t* count);

/* Measured FP32 FMA throughput of CUDA device `device` in TFLOP/s (an FMA
 * counts as two flops): the best of three timed launches of a kernel that
 * runs independent FMA chains on every SM. It is the denominator of the
 * far-field kernels' roofline, which are bound by the FP32 FMA pipe.
 * Library-specific; the paper has no counterpart. Allocates a small device
 * buffer and a stream of its own and synchronises them.
 * Errors: YK_ERR_ARG, YK_ERR_CUDA.                                         */
int yk_fp32_fma_peak(int device, double* tflops);

const char* yk_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* YK_H */
