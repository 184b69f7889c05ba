/*
 * lskum.h -- C ABI of the GB300-native q-LSKUM flux-residual solver.
 *
 * The library solves the steady 2D Euler equations (Eqs. 1-3 of Mamidi et
 * al., "On the performance of GPU accelerated q-LSKUM based meshfree solvers
 * in Fortran, C++, Python, and Julia", 2021) on a meshfree point cloud with
 * the second-order least squares kinetic upwind method in q-variables
 * (Section 2 and Section 2.1, Eqs. 10-29) and the pseudo-time loop of
 * Algorithm 1 / Algorithm 2: per iteration a local time step, four stages of
 * {q-variables, q-derivatives with inner iterations, flux residual, state
 * update} of a four-stage third-order SSP Runge-Kutta scheme, and the residue.
 * Every step runs in hand-written CUDA kernels for sm_103a; there is no CPU
 * fallback: without a usable CUDA device, lskum_create fails.
 *
 * Conventions
 *   - All floating-point arguments are double (FP64) unless stated.
 *   - Point arrays are row-major per point, in the CALLER's point order; the
 *     library reorders points internally (space-filling curve) and maps every
 *     output back to the caller's order.
 *   - Host pointers only (the library owns all device memory it allocates).
 *     Inputs are copied: the caller keeps ownership of its arrays and may
 *     free them after the call returns. Outputs are written into
 *     caller-allocated buffers of the stated size.
 *   - Return value: LSKUM_OK (0) or a negative LSKUM_ERR_* code; no call
 *     throws. lskum_error_string() names a code; lskum_last_error() gives the
 *     detail message of the last failure on this thread.
 *   - A context is used by one host thread at a time. Work is issued on the
 *     context's CUDA stream (lskum_set_stream); calls that return host data
 *     synchronise that stream.
 *   - Primitive state W = (rho, u1, u2, p); conserved state U = (rho, rho u1,
 *     rho u2, rho e) (Eq. 2); residual R of dU/dt + R = 0 (Eq. 12).
 */
#ifndef LSKUM_H
#define LSKUM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LSKUM_OK 0
#define LSKUM_ERR_INVALID_ARG (-1)        /* null pointer, bad size, bad option, n too large */
#define LSKUM_ERR_BAD_CONNECTIVITY (-2)   /* neighbour index out of range, self or repeated
                                             neighbour, offsets not increasing, > 20 neighbours */
#define LSKUM_ERR_DEGENERATE_STENCIL (-3) /* a full or split stencil has a singular 2x2
                                             least-squares matrix (Det <= 1e-12 trace^2) */
#define LSKUM_ERR_CUDA (-4)               /* a CUDA runtime call failed (no device, OOM, ...) */
#define LSKUM_ERR_DIVERGED (-5)           /* non-finite state, rho <= 0 or p <= 0 */
#define LSKUM_ERR_TIMEOUT (-6)            /* a bounded device-side wait gave up */
#define LSKUM_ERR_STATE (-7)              /* call out of order (e.g. step before any state) */

/* Point flags (input). */
#define LSKUM_INTERIOR 0
#define LSKUM_WALL 1  /* solid wall; its normal points into the fluid */
#define LSKUM_OUTER 2 /* far-field boundary; its normal points out of the domain */

#define LSKUM_MAX_NEIGHBOURS 20

/* Precision modes. */
#define LSKUM_FP64 0  /* every step in FP64 */
#define LSKUM_MIXED 1 /* FP32 stencil, least-squares and split-flux arithmetic (in
                         difference form, on q stored as float pairs); FP64 state
                         accumulation, q-variables, LS determinants, residue, forces */

/* Outer-boundary modes. */
#define LSKUM_OUTER_FREESTREAM 1 /* far-field points hold the free-stream state */
#define LSKUM_OUTER_KINETIC 0    /* far-field points updated with dGs+-/ds + dGn+/dn over dn<0 */

typedef struct lskum_ctx lskum_ctx; /* opaque; owned by the library */

typedef struct {
    double gamma;       /* ratio of specific heats (Eq. 3); default 1.4 */
    double cfl;         /* local time step dt_i = cfl min_j d_ij / (|u_i| + a_i); default 0.2 */
    int inner_iters;    /* Jacobi sweeps of Eq. 29 per stage; default 2 (the paper runs 3) */
    int order;          /* 2: q~ defect correction (Eqs. 27-28); 1: first order (Eq. 13) */
    double wall_factor; /* weight of dGn-/dn at wall points; default 2 (specular wall) */
    int outer_mode;     /* LSKUM_OUTER_FREESTREAM (default) or LSKUM_OUTER_KINETIC */
    int precision;      /* LSKUM_FP64 (default) or LSKUM_MIXED */
    int reorder;        /* 1: Hilbert-curve point order on the device (default); 0: input order */
    int block_size;     /* CUDA threads per block of the point kernels; 0 = library default */
    int check_every;    /* lskum_solve: iterations between host convergence checks; default 50 */
    int n_conditions;   /* free streams solved together on the same cloud (a power of two,
                           1..256; default 1). State is laid out condition-innermost on the
                           device; every per-point host array below then holds n_conditions
                           blocks of n points (condition-major), and per-run outputs
                           (residue, Cl, Cd) hold n_conditions values. */
    int flux_split;     /* 0 (default): one fused flux/update kernel per stage. 1: the paper's
                           kernel splitting (Section 5): one kernel per split-flux derivative
                           (dGs+/ds, dGs-/ds, dGn+/dn, dGn-/dn) and one stage-update kernel;
                           an ablation, FP64 only. */
    double weight_power; /* least-squares weights w_j = |P_j - P_i|^-weight_power in every
                           least-squares sum (Eqs. 11, 24, 29), 0 <= weight_power <= 8;
                           default 0: unweighted, as the paper prints them. Applied when the
                           per-neighbour weights are formed at create, so it costs nothing
                           per iteration. */
} lskum_options;

/* Fills *o with the defaults listed above. Returns LSKUM_ERR_INVALID_ARG if o is NULL. */
int lskum_default_options(lskum_options* o);

/*
 * Creates a solver for one point cloud (Section 2: the stencil N(P0) of each
 * point is given by the caller; Eq. 14 split stencils are derived here).
 *   n           number of points, 1 <= n <= 2^26
 *   xy          n x 2 coordinates
 *   normals     n x 2 unit normals; used for wall and outer points (local
 *               frame t = (n_y, -n_x), n); ignored for interior points
 *   flags       n point flags (LSKUM_INTERIOR / LSKUM_WALL / LSKUM_OUTER)
 *   nbr_offsets n + 1 CSR offsets into nbr_idx (nbr_offsets[0] = 0)
 *   nbr_idx     nbr_offsets[n] neighbour indices (0-based, caller's order)
 *   opt         options (NULL: defaults)
 *   out         receives the context; *out is NULL on failure
 * The wall points, in the caller's order, must form closed loops that are
 * walked in index order (the force integral uses consecutive wall points);
 * a loop closes where the next wall point is not a neighbour.
 * Errors: INVALID_ARG, BAD_CONNECTIVITY, DEGENERATE_STENCIL, CUDA.
 */
int lskum_create(int64_t n, const double* xy, const double* normals, const int8_t* flags,
                 const int32_t* nbr_offsets, const int32_t* nbr_idx, const lskum_options* opt,
                 lskum_ctx** out);

/* Frees all device and host memory of the context (NULL is a no-op). */
void lskum_destroy(lskum_ctx* ctx);

/* Issues all later work of ctx on `stream` (a cudaStream_t; NULL = the
 * context's own stream; the legacy default stream is cudaStreamLegacy). The
 * caller keeps the stream alive while in use. */
int lskum_set_stream(lskum_ctx* ctx, void* stream);

/* Free stream rho = 1, p = 1/gamma, u = mach (cos a, sin a), alpha in degrees;
 * also resets the state to the free stream everywhere (the initial condition)
 * and clears the residue history. With n_conditions > 1 every condition gets
 * this free stream. */
int lskum_set_freestream(lskum_ctx* ctx, double mach, double alpha_deg);

/* One free stream per condition (mach[k], alpha_deg[k], k < n_cond; n_cond
 * must equal the context's n_conditions); resets every condition's state to
 * its free stream and clears the residue history. */
int lskum_set_conditions(lskum_ctx* ctx, int n_cond, const double* mach, const double* alpha_deg);

/* Sets the state from n_conditions x n x 4 primitive values (caller's order, host).
 * Errors: INVALID_ARG (null), DIVERGED (non-positive rho or p, non-finite). */
int lskum_set_state(lskum_ctx* ctx, const double* prim);

/* Copies the current primitive state (n_conditions x n x 4, caller's order) to host `prim`. */
int lskum_get_state(lskum_ctx* ctx, double* prim);

/* Runs n_iters pseudo-time iterations of Algorithm 1 on the device (local
 * time step, four SSP-RK stages, residue). Returns DIVERGED if a non-finite
 * or non-positive density/pressure appeared. */
int lskum_step(lskum_ctx* ctx, int n_iters);

/* Iterates until the residue has dropped by `tol` relative to the first
 * non-zero residue of this run (e.g. tol = 1e-6 for six orders) for every
 * condition, or max_iters iterations; *iters_done (may be NULL) receives the
 * count. */
int lskum_solve(lskum_ctx* ctx, int max_iters, double tol, int* iters_done);

/* Residue of the last iteration: sqrt(sum_i R_rho,i^2) / N of its stage-1
 * residual (Algorithm 1, residue()), one value per condition in out[].
 * 0 before the first iteration. */
int lskum_residual_norm(lskum_ctx* ctx, double* out);

/* Lift and drag coefficients of the pressure force on the wall loops:
 * F = -sum (p_i - p_inf) n_i ds_i, Cl/Cd in the free-stream axes, chord 1,
 * q_inf = M^2 / 2; one value per condition in cl[], cd[]. */
int lskum_forces(lskum_ctx* ctx, double* cl, double* cd);

/* Residual R(W) of the current state without updating it: q-variables,
 * q-derivatives (with inner iterations) and flux residual (Eq. 12), written
 * as n_conditions x n x 4 conserved components in the global frame, caller's
 * order. */
int lskum_eval_residual(lskum_ctx* ctx, double* R);

/* q-derivatives (Eq. 11 followed by inner_iters sweeps of Eq. 29) of the
 * current state: qx, qy are n_conditions x n x 4 each, caller's order. */
int lskum_eval_q_derivatives(lskum_ctx* ctx, double* qx, double* qy);

/* Number of points, of wall points in the force loops, the neighbour slots
 * per point of the device layout and the number of conditions (diagnostics;
 * any pointer may be NULL). */
int lskum_info(lskum_ctx* ctx, int64_t* n_points, int64_t* n_wall, int* max_neighbours,
               int* n_conditions);

/* Autotuner: times trial_iters iterations for every pair of thread-block
 * sizes the library is built for (128, 256), one for the flux/update kernel
 * and one for the q-derivative kernels, each from the current state; restores
 * the state, keeps the fastest pair for all later work (re-capturing the
 * iteration graph) and returns it in *best_block as
 * flux_block * 1000 + derivative_block (may be NULL). Clears the residue
 * history. Uses a temporary device buffer of the state's size. */
int lskum_autotune(lskum_ctx* ctx, int trial_iters, int* best_block);

/* Kernel timing with CUDA events on the context's stream, for the roofline
 * report. lskum_profile(ctx, 1) starts recording (clearing old totals), 0
 * stops. lskum_kernel_time(ctx, kernel, &ms, &launches) returns the summed
 * device time and launch count of one kernel class since recording started:
 * kernel 0 flux residual + state update, 1 first-order q-derivatives,
 * 2 inner-iteration q-derivatives, 3 residue/reduction. Timing is exact only
 * when recording is on and CUDA graphs are not used (lskum_step switches to
 * plain launches while recording). */
int lskum_profile(lskum_ctx* ctx, int enable);
int lskum_kernel_time(lskum_ctx* ctx, int kernel, double* total_ms, int64_t* launches);

/* Number of kernel launches issued by the last lskum_step call. */
int64_t lskum_last_launch_count(lskum_ctx* ctx);

/*
 * Residue of a residual the caller already holds, computed without allocating
 * any memory. The paper has no counterpart: this exists for callers that may
 * not allocate device memory at all (code running inside a CUDA-graph capture
 * it does not own, plug-ins whose host framework owns every device allocation,
 * runtimes that forbid allocation after start-up).
 *   R       DEVICE pointer to n x 4 residual values (row-major per point, as
 *           returned by lskum_eval_residual); only R[4 i] (mass) is read
 *   n       number of points, 1 <= n <= LSKUM_NOALLOC_MAX_POINTS
 *   out     DEVICE pointer to one double: sqrt(sum_i R[4 i]^2) / n
 *   stream  cudaStream_t to run on (NULL: the legacy default stream)
 * The kernels keep their per-block partial sums in one fixed 64 KiB array
 * inside the library (8192 partials of 8192 points each); every GPU that
 * loads the library holds that array until the process exits. The first call
 * on each device looks the array's device address up (no allocation); make
 * that first call before any stream capture. The address is kept for the life
 * of the process: after cudaDeviceReset (or any other destruction of the
 * device's primary context) the library's module is loaded again at another
 * address and the kept one is stale, so do not call this entry point on a
 * device after resetting it. All calls on a device share the
 * array and each call overwrites the part it reads, so nothing carries over
 * between calls, but calls that overlap on the GPU (different streams, no
 * ordering between them) race on it. Asynchronous: *out is ready when the
 * stream reaches the end of the call.
 * Errors: INVALID_ARG (null pointer, n out of range; nothing is launched),
 * CUDA (device query or launch failed).
 */
#define LSKUM_NOALLOC_MAX_POINTS (8192LL * 8192LL)
int lskum_residue_noalloc(const double* R, int64_t n, double* out, void* stream);

/* Human-readable name of a return code (static storage). */
const char* lskum_error_string(int code);

/* Detail message of the last failing call on this thread ("" if none). */
const char* lskum_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LSKUM_H */
