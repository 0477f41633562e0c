/*
 * softsim.h -- C ABI of the GB300 (sm_103a) soft-body library.
 *
 * The library evaluates, on one GPU, the hot path of "Differentiable
 * Implicit Soft-Body Physics" (Rojas, Sifakis, Kavan, arXiv 2102.05791):
 * the energy E(x, a) of a triangle / tet mesh (neo-Hookean, Eq.
 * neohookean-psi, plus a per-element muscle term), its gradient (Eq.
 * f-as-grad), its matrix-free Hessian-vector product (Eq. matrix-free-dfdx),
 * the forward minimisation x* = argmin_x E(x, a) (Eq. x1-quasistatic-argmin)
 * or the backward-Euler incremental potential (Eq. opt-be), the adjoint
 * solve H lambda = dL/dx and the parameter VJP dL/da = -lambda^T d2E/dx da
 * (Eq. dLda-re-ordered).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument except those of sim_create is a DEVICE pointer,
 *    allocated and owned by the caller; the library never frees or keeps
 *    it past the call.  Device arrays passed to one call must not overlap
 *    unless stated.
 *  - Vertex fields (positions x, directions v, gradients, lambda) are
 *    row-major [n_vert][dim] (Sec. 3.1 lets x be a 2-D array: vertex, axis).
 *    Axis 1 (y) is vertical; the ground plane is y = 0.
 *  - Element fields (activations a, dL/da) are [n_elem] in the caller's
 *    element order.
 *  - Positions, activations, gradients, lambda and dL/da are double.  The
 *    vectors of sim_hvp are float for SIM_PREC_MIXED and double for
 *    SIM_PREC_FP64.
 *  - `stream` is a cudaStream_t (0 = legacy default stream).  Calls are
 *    stream-ordered; solver calls synchronise the stream internally to read
 *    their convergence scalars and return only when their outputs are
 *    written.
 *  - Return value: SIM_OK (0) or a negative SIM_E* code.  Nothing aborts;
 *    sim_last_error() gives a message.  A handle is not thread-safe: calls
 *    on one handle must not run concurrently.
 *  - Pinned (Dirichlet) vertices: gradient, HVP, lambda and search
 *    directions are zero there, and x_init must hold their rest position.
 */
#ifndef SOFTSIM_H
#define SOFTSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SIM_OK = 0,
    SIM_EINVAL = -1,          /* bad argument */
    SIM_ECUDA = -2,           /* CUDA runtime error */
    SIM_EINVERTED = -3,       /* element with non-positive rest volume, or x inverts one */
    SIM_ENOTCONVERGED = -4,   /* iteration cap reached */
    SIM_ELINESEARCH = -5,     /* no step length met the descent condition */
    SIM_ENAN = -6,            /* non-finite value in the inputs or the iterates */
    SIM_ENOMEM = -7           /* device allocation failed */
};

enum { SIM_PREC_FP64 = 0, SIM_PREC_MIXED = 1 };
enum { SIM_LOG_EXACT = 0, SIM_LOG_QUAD = 1 };
enum { SIM_MUSCLE_CONTRACTILE = 0, SIM_MUSCLE_SPRING = 1 };
enum { SIM_CG_AUTO = 0, SIM_CG_ITERATION = 1 };

typedef struct sim_handle sim_handle;

/* Mesh, given in HOST memory and copied by sim_create. */
typedef struct {
    int dim;                  /* 2 (triangles) or 3 (tetrahedra) */
    int64_t n_vert, n_elem;
    const double *rest_pos;   /* [n_vert][dim] rest positions X */
    const int32_t *elems;     /* [n_elem][dim+1] vertex ids, 0 <= id < n_vert */
    const uint8_t *fixed;     /* [n_vert] 1 = pinned vertex, or NULL for none */
} sim_mesh;

/* Material (Sec. 2 and 4): E(x,a) = sum_e W_e [Psi(F_e) + k/2 a_e |F_e f_e|^2]
 *   + sum_i m_i g y_i + sum_i k_c max(0, -y_i)^p, with
 *   Psi = mu/2 (tr F^T F - dim) - mu l(J) + lambda/2 l(J)^2,
 *   l = log (SIM_LOG_EXACT; E = +inf if some J <= 0) or
 *   l(J) = (J-1) - (J-1)^2/2 (SIM_LOG_QUAD, the quadratic stand-in of Sec. 2),
 *   W_e the rest area / volume, m_i = sum over elements of rho W_e/(dim+1).
 * dt > 0 selects backward Euler (Eq. opt-be): the solver then minimises
 *   1/2 |x - (x0 + dt v0)|_M^2 + dt^2 E(x, a).
 * k_friction > 0 (dynamics only; ignored when dt == 0) adds the ground
 * friction of Sec. 4.2, dt^2 sum_i k_f |v_h,i|^2 ReLU(eps_friction - y0_i),
 * with v = (x - x0)/dt and v_h its horizontal part (every axis but y): the
 * damping acts on vertices that started the step within eps_friction of
 * the ground (or below it).  A zero-initialised struct has friction off.
 * muscle_model selects psi_m: SIM_MUSCLE_CONTRACTILE (k/2) a |F f|^2, or
 * SIM_MUSCLE_SPRING (k/2)(|F f|/a - 1)^2, the active spring of Eq.
 * active-spring-potential with |F f| = l/l0 the fiber stretch; it needs
 * a > 0 (a <= 0 makes the energy non-finite: SIM_ENAN). */
typedef struct {
    double mu, lambda;        /* Lame parameters */
    double k_muscle;          /* muscle stiffness k */
    double density;           /* rho, for the lumped mass */
    double gravity;           /* g along -y */
    double k_contact;         /* ground penalty stiffness k_c (0 = off) */
    int contact_power;        /* p = 2 (Eq. energy-collision) or 3 */
    int log_mode;             /* SIM_LOG_EXACT or SIM_LOG_QUAD */
    double dt;                /* 0 = quasistatic; > 0 = backward-Euler step */
    const double *fiber;      /* HOST [n_elem][dim] unit fiber directions */
    double k_friction;        /* ground friction stiffness k_f (0 = off) */
    double eps_friction;      /* height below which friction acts */
    int muscle_model;         /* SIM_MUSCLE_CONTRACTILE (0) or SIM_MUSCLE_SPRING */
} sim_material;

typedef struct {
    int precision;            /* SIM_PREC_FP64 (all FP64) or SIM_PREC_MIXED
                                 (FP32 HVP and CG vectors; FP64 state, gradient,
                                 energy, reductions and residual checks) */
    double newton_rtol;       /* stop when |grad| <= newton_rtol |grad_0| */
    double newton_forcing;    /* cap of the CG forcing term: each Newton step's CG
                                 stops at |r| <= min(newton_forcing,
                                 sqrt(|g|/|g0|)) |g| */
    double adjoint_rtol;      /* adjoint CG: stop when |r| <= adjoint_rtol |b| */
    int max_newton;           /* Newton iteration cap */
    int max_cg;               /* CG iteration cap per Newton step */
    int max_adjoint_cg;       /* CG iteration cap of the adjoint solve */
    int max_ls;               /* backtracking halvings cap */
    int tile_elems;           /* elements per tile (0 = library default) */
    int threads;              /* threads per element-kernel block (0 = default) */
    int cg_kernel;            /* SIM_CG_AUTO: a whole CG solve in one kernel when
                                 every tile of the mesh fits on the GPU at once (one
                                 thread-block cluster for at most 16 tiles, else a
                                 cooperative grid), else per-iteration kernels;
                                 SIM_CG_ITERATION: always per-iteration kernels */
} sim_options;

typedef struct {
    int newton_iters;         /* Newton steps taken */
    int cg_iters_total;       /* CG iterations over all steps */
    int ls_halvings;          /* total backtracking halvings */
    int status;               /* SIM_OK or SIM_E* of the solve */
    double res0, res_final;   /* FP64 |grad| (forward) or |r| (adjoint), first and last */
    double min_J;             /* smallest det F at the returned state */
} sim_solve_stats;

/* Fill `opt` with the defaults (MIXED, rtol 1e-8, forcing cap 0.5, adjoint
 * 1e-6, 100 Newton, 500 CG, 4 n_dof adjoint CG cap, 30 halvings,
 * SIM_CG_AUTO). */
int sim_default_options(sim_options *opt);

/* Build a handle: validates the mesh (ids in range, positive rest volumes),
 * computes Dm^-1, W_e and lumped masses, orders elements into tiles for the
 * deterministic vertex scatter, and uploads everything.  All pointers are
 * HOST pointers and are copied.  On failure *out is NULL and the message is
 * available from sim_last_error(NULL). */
int sim_create(const sim_mesh *mesh, const sim_material *mat, const sim_options *opt,
               sim_handle **out);

/* Free the handle and every device buffer it owns. */
int sim_destroy(sim_handle *h);

/* Last error message of the handle (or of the last failed sim_create when h
 * is NULL).  The string lives until the next call on the handle. */
const char *sim_last_error(const sim_handle *h);

/* Sizes of the handle's mesh: dim, n_vert, n_elem. */
int sim_sizes(const sim_handle *h, int *dim, int64_t *n_vert, int64_t *n_elem);

/* E(x, a) and grad_x E (Eq. f-as-grad, f = -grad), FP64, quasistatic energy
 * (no inertia term even when dt > 0).  E_dev: one double on the device, or
 * NULL; grad: [n_vert][dim] double, zero at pinned vertices, or NULL.
 * E is +inf when SIM_LOG_EXACT and some element has J <= 0. */
int sim_energy_grad(sim_handle *h, const double *x, const double *a, double *E_dev,
                    double *grad, void *stream);

/* Hv = H(x, a) v, the Hessian of the quasistatic E applied to v (Eq.
 * matrix-free-dfdx), with pinned rows and columns dropped.  v and Hv are
 * [n_vert][dim] float (MIXED) or double (FP64); x, a double. */
int sim_hvp(sim_handle *h, const double *x, const double *a, const void *v, void *Hv,
            void *stream);

/* The CG loop's inner product v.(H v) (Eq. matrix-free-dfdx), formed as the
 * CG loop forms p.Ap: each element's quadratic form v_e.(H_e v_e) plus the
 * per-vertex terms, summed in FP32 within a tile and with compensated FP32
 * over the tiles (SIM_PREC_MIXED), or in FP64 throughout (SIM_PREC_FP64).
 * Diagnostic, to measure that sum's error.  v, Hv: DEVICE [n_vert][dim] in
 * the HVP precision (as for sim_hvp; Hv receives H v); x, a: DEVICE double;
 * *vHv: HOST double.  Synchronises the stream. */
int sim_hvp_dot(sim_handle *h, const double *x, const double *a, const void *v, void *Hv, double *vHv,
                void *stream);

/* Forward solve.  Quasistatic (dt == 0): x_out = argmin_x E(x, a) (Eq.
 * x1-quasistatic-argmin), started from x_init; x0 and v0 must be NULL.
 * Backward Euler (dt > 0): x_out = argmin 1/2 |x - (x0 + dt v0)|_M^2 +
 * dt^2 E(x, a) (Eq. opt-be), started from x_init (NULL = x0).  Newton-CG with
 * forcing eta = min(0.5, sqrt(|g|/|g0|)), backtracking line search with the
 * Armijo constant 1e-4 on FP64 energies, rejecting inverted elements under
 * the exact log.  `stats` may be NULL.  x_out may alias x_init. */
int sim_newton_solve(sim_handle *h, const double *x_init, const double *a, const double *x0,
                     const double *v0, double *x_out, sim_solve_stats *stats, void *stream);

/* Adjoint solve at a converged state (Eq. dLda-re-ordered): lambda =
 * A^-1 b with A = H(x*, a) (quasistatic) or M + dt^2 H(x*, a) (backward
 * Euler), b = dLdx with pinned entries dropped; CG to adjoint_rtol.  With
 * friction, A uses the friction weights of the last step prepared by
 * sim_newton_solve / sim_step_forward / sim_step_backward. */
int sim_adjoint_solve(sim_handle *h, const double *x_star, const double *a, const double *dLdx,
                      double *lambda, sim_solve_stats *stats, void *stream);

/* Parameter VJP (Eq. dLda-re-ordered): dLda_e = -s lambda^T d(grad E)/da_e
 * = -s W_e (d2psi_m/dq da) . (dF_e(lambda) f_e) with q = F_e f_e, i.e.
 * k q for the contractile muscle and k (1/a^2 - 2|q|/a^3) q/|q| for the
 * spring; s = dt^2 for backward Euler and 1 otherwise.  a: DEVICE
 * [n_elem] activations at which x_star was solved.  Output [n_elem] double
 * in the caller's element order. */
int sim_param_vjp(sim_handle *h, const double *x_star, const double *a, const double *lambda,
                  double *dLda, void *stream);

/* Material-parameter VJPs per element (Eq. dLda-re-ordered with a material
 * parameter theta in place of a): dL/dtheta_e = -s lambda^T d(grad E)/dtheta_e
 * = -s W_e (dP_e/dtheta) : dF_e(lambda) for theta = mu, lambda, with
 * dP/dmu = F - l'(J) cof F and dP/dlambda = l(J) l'(J) cof F (l the exact or
 * quadratic log), and -s W_e (d2psi_m/dq dk) . (dF_e(lambda) f_e) for the
 * muscle stiffness k.  The derivative for a global parameter (or one mesh's)
 * is the sum over elements.  x_star, a, lambda as for sim_param_vjp; each
 * output is a DEVICE [n_elem] double array in the caller's element order, or
 * NULL to skip it. */
int sim_material_vjp(sim_handle *h, const double *x_star, const double *a, const double *lambda,
                     double *dLdmu, double *dLdlambda, double *dLdk, void *stream);

/* One backward-Euler step (Eq. opt-be), dt > 0 only: x1 = argmin of the
 * incremental potential started from x0, v1 = (x1 - x0)/dt.  x1 and v1 must
 * not alias x0 or v0. */
int sim_step_forward(sim_handle *h, const double *x0, const double *v0, const double *a,
                     double *x1, double *v1, sim_solve_stats *stats, void *stream);

/* Backward of one backward-Euler step, given the step's inputs and its
 * result x1 and the loss gradients xbar1 = dL/dx1, vbar1 = dL/dv1:
 *   lambda = (M + dt^2 H(x1))^-1 (xbar1 + vbar1/dt),
 *   xbar0 = M lambda - vbar1/dt,  vbar0 = dt M lambda,
 *   abar = -dt^2 lambda^T d2E/dx da.
 * With friction, H includes its horizontal stiffness fw_i = 2 k_f ReLU(eps -
 * y0_i) and xbar0 gains fw_i lambda_h,i on the horizontal axes and
 * 2 k_f [y0_i < eps] lambda_h,i . (x1 - x0)_h,i on y; x0 is then required
 * (v0 is never read).
 * Outputs may not alias inputs; xbar0/vbar0 are zero at pinned vertices. */
int sim_step_backward(sim_handle *h, const double *x0, const double *v0, const double *x1,
                      const double *a, const double *xbar1, const double *vbar1, double *xbar0,
                      double *vbar0, double *abar, sim_solve_stats *stats, void *stream);

/* Rollout of n_steps backward-Euler steps from (x0, v0) with activations
 * a_seq [n_steps][n_elem].  Writes the final state to xT, vT and, every
 * ckpt_every steps (t = 0, ckpt_every, 2 ckpt_every, ... < n_steps), the
 * state (x_t, v_t) to ckpt_x / ckpt_v [n_ckpt][n_vert][dim], n_ckpt =
 * ceil(n_steps / ckpt_every).  `stats` (may be NULL) accumulates over steps. */
int sim_rollout(sim_handle *h, int n_steps, const double *x0, const double *v0, const double *a_seq,
                int ckpt_every, double *ckpt_x, double *ckpt_v, double *xT, double *vT,
                sim_solve_stats *stats, void *stream);

/* Backpropagation through time over a checkpointed rollout: recomputes each
 * segment from its checkpoint into the caller's work buffers seg_x, seg_v
 * [ckpt_every + 1][n_vert][dim] and runs sim_step_backward in reverse.
 * Inputs xbarT, vbarT = dL/dx_T, dL/dv_T; outputs xbar0, vbar0 and
 * abar_seq [n_steps][n_elem]. */
int sim_rollout_backward(sim_handle *h, int n_steps, const double *a_seq, int ckpt_every,
                         const double *ckpt_x, const double *ckpt_v, const double *xbarT,
                         const double *vbarT, double *xbar0, double *vbar0, double *abar_seq,
                         double *seg_x, double *seg_v, sim_solve_stats *stats, void *stream);

/* Kernel timer: launches the element HVP kernel n_launches times back to
 * back on the handle's current internal state (after a solve) on `stream`
 * and writes the mean duration of one launch, in milliseconds, measured with
 * CUDA events, for the tile kernel (ms[0]) and the halo-finalise kernel
 * (ms[1]).  Back-to-back launches can find part of the previous launch's
 * data in L2; sim_kernel_timing measures launches inside a solve. */
int sim_time_hvp(sim_handle *h, int n_launches, float *ms, void *stream);

/* In-solve kernel timing.  When switched on, the CG iterations of later
 * solves record CUDA events around every HVP tile-kernel launch (on the
 * launching stream, inside the captured graphs); sim_kernel_timing returns
 * the summed duration in milliseconds and the number of timed launches since
 * timing was last switched on (switching resets both). */
int sim_set_kernel_timing(sim_handle *h, int on);
int sim_kernel_timing(const sim_handle *h, double *hvp_tile_ms, int64_t *hvp_launches);

/* Poll limit of the first bulk-copy wait in the HVP tile kernels (the wait
 * for a tile's vertex tables), for testing the timeout path: polls >= 0 sets
 * it (0 = give up at once), polls < 0 restores the library default (the
 * bound of every other wait).  A kernel whose wait runs out raises a flag,
 * lets the copies it issued land, and exits without touching the unfinished
 * data; the solver call that launched it then returns SIM_ECUDA ("gave up
 * waiting") and clears the flag, so the handle's next call starts clean. */
int sim_set_wait_limit(sim_handle *h, int polls);

/* Number of CUDA kernels the handle has launched so far (graph replays count
 * every kernel node they run). */
int sim_counters(const sim_handle *h, int64_t *kernel_launches);

/* Tiling statistics: n_tiles, mean elements per tile, mean local vertices
 * per tile, fraction of vertices shared between tiles. */
int sim_tile_stats(const sim_handle *h, int *n_tiles, double *elems_per_tile,
                   double *verts_per_tile, double *halo_fraction);

/* ---------------------------------------------------------------- batches
 * Many independent meshes of uneven size (same dim; materials, ground
 * friction included, may differ only in mu and lambda), each rolled out for
 * n_steps backward-Euler steps (Eq. opt-be) and differentiated by backpropagation through time, in ONE
 * persistent kernel launch replayed from a captured CUDA graph.  Each CTA
 * takes the next mesh (largest first) and runs its whole forward rollout
 * (Newton-CG per step) and backward pass (refined adjoint CG and parameter
 * VJP per step, Eq. dLda-re-ordered) with block-level synchronisation only.
 * Mixed precision as SIM_PREC_MIXED.  Deterministic: a mesh is always
 * computed by one CTA with a fixed thread count and fixed-order sums. */
typedef struct sim_batch sim_batch;

/* Meshes, materials (dt > 0) and options as for sim_create, HOST arrays,
 * copied.  Vertices and elements of mesh m follow those of meshes 0..m-1 in
 * every concatenated array below. */
int sim_batch_create(int n_meshes, const sim_mesh *meshes, const sim_material *mats,
                     const sim_options *opt, sim_batch **out);
int sim_batch_destroy(sim_batch *b);
const char *sim_batch_last_error(const sim_batch *b);
int sim_batch_sizes(const sim_batch *b, int *n_meshes, int64_t *total_vert, int64_t *total_elem);

/* Forward rollout and BPTT of every mesh.  DEVICE arrays, V/E = total
 * vertices/elements, d = dim:
 *   states_x, states_v [n_steps+1][V][d]: slot 0 holds the initial state on
 *     entry; slots 1..n_steps receive the states x_t, v_t;
 *   a_seq [n_steps][E] activations per step;
 *   xbarT, vbarT [V][d] = dL/dx_T, dL/dv_T;
 *   abar_seq [n_steps][E] receives dL/da_t; xbar0, vbar0 [V][d] receive
 *     dL/dx_0, dL/dv_0;
 *   mesh_stats [n_meshes][4] ints (or NULL): status, Newton iterations, CG
 *     iterations forward, CG iterations adjoint;
 *   mat_grad [n_meshes][3] doubles (or NULL): dL/dmu_m, dL/dlambda_m and
 *     dL/dk of mesh m, summed over its elements and steps (the material VJP
 *     of sim_material_vjp at each step's lambda, dt^2-scaled); for the shared
 *     k the batch's derivative is the sum over meshes.
 * Stream-ordered; returns after enqueueing (synchronise before reading). */
int sim_batch_rollout(sim_batch *b, int n_steps, double *states_x, double *states_v,
                      const double *a_seq, const double *xbarT, const double *vbarT,
                      double *abar_seq, double *xbar0, double *vbar0, int *mesh_stats,
                      double *mat_grad, void *stream);

/* Energy without allocation.  The paper has no counterpart: this is a
 * deployment aid.  Returns in E_out (one device double) the quasistatic
 * energy E(x, a) of sim_energy_grad for a mesh given entirely as
 * caller-owned DEVICE arrays -- rest_pos, x [n_vert][dim] double, elems
 * [n_elem][dim+1] int32, a [n_elem] double, fiber [n_elem][dim] double --
 * with the scalars of `mat` (a host struct; its fiber and dt fields are
 * ignored).  It needs no handle and allocates no device memory, for callers
 * that cannot call cudaMalloc at that point: a process whose GPU memory is
 * already claimed by another framework's pool allocator, or code that must
 * not allocate after its setup.  Its scratch (block partial sums and two
 * counters, about 33 KB) is a fixed array inside the library that every GPU
 * loading the library keeps until exit.  At most 4,194,304 elements and
 * vertices; larger meshes get SIM_EINVAL.  The first call on a device looks
 * up the array's address (with that device current) and must come before
 * any stream capture.  Calls share the array, so calls that overlap on the
 * GPU race; serialise them.  The call waits for `stream` before it returns:
 * a rest element with non-positive area or volume (which sim_create would
 * reject) gives SIM_EINVERTED, with E_out = NaN.  Under SIM_LOG_EXACT a
 * state with some J <= 0 gives E = +inf and SIM_OK, as in sim_energy_grad.
 * Errors: sim_noalloc_last_error(). */
int sim_energy_noalloc(int dim, int64_t n_vert, int64_t n_elem, const double *rest_pos,
                       const int32_t *elems, const double *x, const double *a, const double *fiber,
                       const sim_material *mat, double *E_out, void *stream);
const char *sim_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SOFTSIM_H */
