/*
 * mba.h -- C ABI of the GB300 bundle-adjustment library (one GPU, sm_103a).
 *
 * The library runs the hot path of the MegBA method (arXiv 2112.01349): one
 * Levenberg-Marquardt iteration over BAL cameras and 3-D points is
 *   residual + analytic Jacobian per observation        (Alg. 1, Jacobian step)
 *   Hessian blocks B, C, E and gradient v, w             (Sec. 3 Eq. 2; Alg. 1)
 *   Schur elimination of the points                      (Sec. 3 Eq. 3)
 *   block-Jacobi PCG on the reduced camera system with
 *   the implicit Schur product                           (Alg. 2, Alg. 3)
 *   point back-substitution                              (Sec. 3 Eq. 4)
 *   additive update and trust-region accept/reject       (Alg. 1; supplement)
 * The paper's edge partitioning across GPUs and its allreduces collapse to
 * the identity on one GPU and are not part of this interface.
 *
 * Conventions for every function:
 *  - Pointers named in the argument lists are HOST pointers unless stated.
 *    Inputs are copied; the library never keeps a caller pointer.
 *  - Camera arrays are nc x 9 row-major doubles in BAL order
 *    (angle-axis w[3], translation t[3], focal f, radial k1, k2); point arrays
 *    np x 3; observation arrays n x 2 pixels; index arrays are int32.
 *  - Functions return an mba_status and never abort or print.  On failure,
 *    mba_last_error() describes the cause (per calling thread).
 *  - A problem handle owns all of its device memory, sized once at creation;
 *    no call after mba_problem_create allocates device memory.  Handles are not
 *    thread-safe; separate handles are independent.
 *  - All work is issued on the stream given at creation and every call
 *    returns after that stream has finished the call's work.
 */
#ifndef MBA_H
#define MBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mba_problem mba_problem;

typedef enum {
    MBA_OK = 0,
    MBA_ERR_INVALID_ARG = 1,   /* bad size, index out of range, unsupported shape */
    MBA_ERR_OOM = 2,           /* device allocation failed at creation */
    MBA_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    MBA_ERR_NONFINITE = 4,     /* non-finite input, or a damped block is not positive definite */
    MBA_ERR_TIMEOUT = 5,       /* a grid-wide barrier of the persistent solver gave up waiting */
    MBA_ERR_NOT_CONVERGED = 6  /* reserved */
} mba_status;

typedef enum { MBA_FP64 = 0, MBA_FP32_MIXED = 1 } mba_precision;
typedef enum { MBA_LOSS_NONE = 0, MBA_LOSS_HUBER = 1 } mba_loss;
/* Damping: DIAG adds mu * clamp(diag(H), 1e-6, 1e32) (the Ceres trust-region form the
 * supplement names); IDENTITY adds mu * I (the form written in Sec. 3). */
typedef enum { MBA_DAMP_DIAG = 0, MBA_DAMP_IDENTITY = 1 } mba_damping;
/* PCG preconditioner.  BLOCK_JACOBI: M = blockdiag(B~_i), as Alg. 2 writes it (default).
 * SCHUR_JACOBI (solver variant, not in the paper): M = blockdiag(S~_ii) with
 * S~_ii = B~_i - sum over the observations k of camera i of E_k C~^-1 E_k^T, the exact
 * diagonal blocks of S when each (camera, point) pair is observed once; a block that is
 * not positive definite falls back to B~_i.  Inverted in FP64 in both forms. */
typedef enum { MBA_PRECOND_BLOCK_JACOBI = 0, MBA_PRECOND_SCHUR_JACOBI = 1 } mba_preconditioner;

/* Source of the residuals and Jacobians (Sec. 3.2).  ANALYTIC: the hand-derived chain
 * rule of the BAL camera (the paper's "-m" form, default).  AUTODIFF: the edge is
 * written once as a functor over a generic scalar and evaluated on forward-mode
 * dual numbers (mba_jet.cuh), which yields the value and both Jacobian blocks (the
 * paper's "-a" form).  Both give the same Jacobian up to rounding; AUTODIFF costs
 * more arithmetic per linearisation and, in FP32_MIXED, an extra stored camera-major
 * Jacobian (72 bytes per observation) for the PCG camera pass. */
typedef enum { MBA_JACOBIAN_ANALYTIC = 0, MBA_JACOBIAN_AUTODIFF = 1 } mba_jacobian;

/* Arithmetic of the cost F(x) and F(x + dx) that decides LM accept/reject (Alg. 1;
 * supplement, trust region).  FP64 (default): every residual and the sum in FP64.
 * FLOAT_FLOAT (option of the FP32-mixed analytic form only; other problems ignore it
 * and keep FP64): residuals and sums in float-float arithmetic (pairs of floats,
 * about 48 significant bits, Dekker's and Knuth's error-free transformations) on the
 * FP32 pipe, which is faster than the FP64 pipe; its relative error per residual is
 * about 1e-13, so accept/reject decisions can differ from FP64 only where the gain
 * ratio sits within that of the acceptance threshold. */
typedef enum { MBA_COST_FP64 = 0, MBA_COST_FLOAT_FLOAT = 1 } mba_cost_arithmetic;

/* Recurrence of the PCG (Alg. 2).  STANDARD (default): the loop as Alg. 2 writes it,
 * two inner-product reductions per iteration (p.q for alpha, r.z for beta).
 * SINGLE_REDUCTION (solver variant, not in the paper): the one-step method of
 * Chronopoulos and Gear (J. Comput. Appl. Math. 25, 1989): with u = M^-1 r and
 * w = S u, the products r.u, w.u and r.r are taken together after the Schur product,
 * alpha = r.u / (w.u - beta r.u / alpha_prev), and s = S p follows by the recurrence
 * s = w + beta s.  The iterates equal the standard ones in exact arithmetic; the
 * persistent PCG kernel then needs one global reduction per iteration instead of two,
 * and three grid barriers per iteration where the standard loop needs three (search
 * direction in shared memory) or four.  The iteration count and stopping test are
 * unchanged; a solve that meets the tolerance forms one Schur product more than it
 * uses. */
typedef enum { MBA_PCG_STANDARD = 0, MBA_PCG_SINGLE_REDUCTION = 1 } mba_pcg_variant;

typedef struct {
    int32_t precision;   /* mba_precision.  FP32_MIXED: Jacobian, Hessian blocks and the
                            PCG Schur product in FP32; block inversions, PCG dot
                            products and norms, cost and accept/reject in FP64. */
    int32_t loss;        /* mba_loss; cost F = 1/2 sum rho(|e|^2) (Eq. 1 with Sigma = I) */
    double huber_delta;  /* Huber threshold in pixels (MBA_LOSS_HUBER) */
    void *cuda_stream;   /* cudaStream_t to run on; NULL = the legacy default stream */
    int32_t jacobian;    /* mba_jacobian (default ANALYTIC); batches accept ANALYTIC only */
    int32_t pad;
} mba_problem_options;

typedef struct {
    int32_t max_iter;              /* LM iterations (rejected ones count) */
    int32_t pcg_max_iter;          /* PCG iteration cap per LM iteration (Alg. 2) */
    double pcg_rel_tol;            /* stop PCG when |r|_2 <= tol * |r0|_2 */
    int32_t damping;               /* mba_damping */
    double initial_radius;         /* trust-region radius; mu = 1 / radius */
    double min_relative_decrease;  /* accept a step iff gain ratio > this */
    double function_tol;           /* > 0: stop after an accepted step with |dF|/F < tol; 0: run max_iter */
    int64_t barrier_spin_limit;    /* polls before a grid barrier gives up (MBA_ERR_TIMEOUT); 0 = default */
    int32_t collect_timing;        /* 1: fill the ms_* fields of mba_summary with CUDA-event times */
    int32_t preconditioner;        /* mba_preconditioner (default BLOCK_JACOBI) */
    int32_t forcing;               /* 1: inexact-Newton forcing sequence (solver variant): each solve's
                                      PCG tolerance is max(pcg_rel_tol, min(0.1, sqrt(|g|/|g_1|))), |g| the
                                      norm of its reduced right-hand side, |g_1| that of the solve's first
                                      damped step; 0: pcg_rel_tol throughout (default) */
    int32_t cost_arithmetic;       /* mba_cost_arithmetic (default FP64) */
    int32_t pcg_variant;           /* mba_pcg_variant (default STANDARD) */
} mba_solver_options;

/* One LM iteration as recorded by mba_solve. */
typedef struct {
    double cost;              /* F(x) before the iteration */
    double cost_new;          /* F(x + dx) of the candidate */
    double model_decrease;    /* 1/2 sum W_k (|e_k|^2 - |e_k + J_k dx|^2) */
    double mu;                /* damping used */
    double gain;              /* (cost - cost_new) / model_decrease */
    int32_t accepted;
    int32_t pcg_iters;
    double pcg_rel_residual;  /* |r|_2 / |r0|_2 at PCG exit */
} mba_iteration;

typedef struct {
    int32_t iterations;        /* LM iterations run */
    int32_t accepted;          /* accepted steps */
    int32_t pcg_iters_total;
    int32_t status;            /* mba_status of the solve */
    double initial_cost, final_cost;
    double final_mu;           /* 1 / final radius */
    double final_radius;
    double ms_total;           /* device time of the whole solve (collect_timing) */
    double ms_linearize;       /* residual/Jacobian/Hessian-block kernels */
    double ms_pcg;             /* persistent PCG kernel (incl. Schur right-hand side) */
    double ms_other;           /* damping, back-substitution, cost, LM control */
    int32_t kernel_launches;   /* CUDA kernels this solve launched (gated-off ones included) */
    mba_iteration *trace;      /* optional caller buffer of trace_capacity entries (host) */
    int32_t trace_capacity;
} mba_summary;

/* Defaults: FP64, no loss, delta 0, default stream / max_iter 10, pcg_max_iter 100,
 * pcg_rel_tol 1e-10, DIAG damping, radius 1e4, min decrease 1e-3, function_tol 0,
 * FP64 accept/reject cost. */
void mba_problem_options_default(mba_problem_options *opt);
void mba_solver_options_default(mba_solver_options *opt);

/*
 * Create a problem: copy cameras (nc x 9), points (np x 3), observations
 * (n x 2) with cam_idx[n], pt_idx[n] to the device, validate them, sort the
 * observations stably by point and by camera (the CSR layout of E and E^T,
 * Sec. 4.1) and size every buffer the solver will use (Sec. 5.2, buffers
 * sized once).  Errors: MBA_ERR_INVALID_ARG for nc, np or n < 1, n >= 2^31,
 * an index out of range, a camera or point without observations, or a point
 * seen more than 1024 times; MBA_ERR_NONFINITE for a NaN/Inf input;
 * MBA_ERR_OOM, MBA_ERR_CUDA.  *out is NULL on failure.
 */
mba_status mba_problem_create(const double *cameras, int32_t nc, const double *points, int32_t np,
                              const double *observations, const int32_t *cam_idx, const int32_t *pt_idx,
                              int64_t n, const mba_problem_options *opt, mba_problem **out);

void mba_problem_destroy(mba_problem *problem);

/* Sizes and the device memory the handle owns. */
mba_status mba_problem_info(const mba_problem *problem, int32_t *nc, int32_t *np, int64_t *n,
                            size_t *device_bytes);

/*
 * Cost F = 1/2 sum_k rho(|e_k|^2) (FP64) at the current parameters and, for
 * each non-NULL output, the raw (unweighted) residuals e_k = pi(c_i, X_j) - u_k
 * (n x 2), camera Jacobians (n x 2 x 9) and point Jacobians (n x 2 x 3), in the
 * caller's observation order, computed in the problem's precision (Alg. 1,
 * residual/Jacobian step).
 */
mba_status mba_evaluate(mba_problem *problem, double *cost, double *residuals, double *jac_cam,
                        double *jac_pt);

/* Run the LM solve (Alg. 1 loop) from the current parameters. */
mba_status mba_solve(mba_problem *problem, const mba_solver_options *opt, mba_summary *summary);

/* Copy the current parameters out / in (host arrays nc x 9 and np x 3). */
mba_status mba_get_parameters(const mba_problem *problem, double *cameras, double *points);
mba_status mba_set_parameters(mba_problem *problem, const double *cameras, const double *points);
/* Restore the parameters given at creation (device-to-device). */
mba_status mba_reset(mba_problem *problem);

/*
 * Hold cameras and points constant, as the fixed vertices of the g2o / Ceres
 * graph convention that the paper's API follows (Sec. 5.3).  cam_fixed (nc
 * bytes) and pt_fixed (np bytes) are host arrays; a nonzero byte marks a node
 * fixed; NULL means none of that kind is fixed (so mba_set_fixed(p, NULL, NULL)
 * clears every mark).  A fixed node's Jacobian columns are taken as zero in
 * every solve-side computation: its Hessian block and gradient vanish, it has no
 * Schur coupling, its step (mba_step, mba_solve) is exactly zero and it stays
 * bit-identical; its initial-estimate gradient (mba_adjoint) is the upstream
 * gradient and it contributes nothing to the observation gradient.
 * mba_evaluate still reports the model's full Jacobians.  The marks persist
 * until the next call.  Errors: MBA_ERR_INVALID_ARG for a NULL problem,
 * MBA_ERR_CUDA.
 */
mba_status mba_set_fixed(mba_problem *problem, const uint8_t *cam_fixed, const uint8_t *pt_fixed);

/*
 * The stable orderings built at creation: pt_perm[n] lists observation indices
 * grouped by point (increasing index within a point), pt_ptr[np + 1] its CSR
 * offsets; cam_perm / cam_ptr likewise by camera.  Any output may be NULL.
 */
mba_status mba_get_ordering(const mba_problem *problem, int32_t *pt_perm, int32_t *pt_ptr, int32_t *cam_perm,
                            int32_t *cam_ptr);

/*
 * Linearise at the current parameters with damping mu and copy out the
 * undamped blocks: Hpp (nc x 9 x 9) = B, v (nc x 9), Hll (np x 3 x 3) = C,
 * w (np x 3) (Eq. 2, built as in Alg. 1), and the reduced-camera right-hand
 * side rhs (nc x 9) = v - E C~^-1 w with C~ damped (Eq. 3).  Any output may be NULL.
 */
mba_status mba_linear_system(mba_problem *problem, double mu, int32_t damping, double *Hpp, double *v,
                             double *Hll, double *w, double *rhs);

/* y = S x with S = B~ - E C~^-1 E^T at damping mu, applied implicitly (Alg. 3);
 * x and y are nc x 9. */
mba_status mba_schur_matvec(mba_problem *problem, double mu, int32_t damping, const double *x, double *y);

/*
 * One damped step at the current parameters: PCG on the reduced camera system
 * (Alg. 2, with opt->pcg_max_iter / pcg_rel_tol / damping) and point
 * back-substitution (Eq. 4).  Outputs: dc (nc x 9), dp (np x 3), the PCG
 * iteration count and the linear model decrease; any may be NULL.
 * The parameters are not changed.
 */
mba_status mba_step(mba_problem *problem, double mu, const mba_solver_options *opt, double *dc, double *dp,
                    int32_t *pcg_iters, double *model_decrease);

/*
 * Gradient of the solved state for a differentiable BA layer (the paper has
 * no counterpart; it reuses the Schur elimination and PCG of Alg. 2/3).  At
 * the current parameters x* (normally the result of mba_solve), with
 * M = H(x*) + mu D the damped Gauss-Newton matrix, v = M^-1 gbar is found by
 * Schur elimination, PCG (opt->pcg_max_iter, opt->pcg_rel_tol, opt->damping)
 * and back-substitution, gbar = (grad_cameras nc x 9, grad_points np x 3) being
 * dL/dx*.  By the implicit function theorem on J^T W e = 0:
 *   grad_obs (n x 2, caller's order)  dL/du_k = W_k J_k v
 *   grad_init_cam (nc x 9), grad_init_pt (np x 3)  dL/dx0 = mu D v, the initial
 *     estimate entering through the damping of the last (proximal) LM step.
 * mu < 0 takes the damping of the last accepted step of the last mba_solve
 * (the proximal step that produced x*); the exact implicit-function gradient
 * of the observations is the limit mu -> 0, so a small explicit mu gives it
 * more closely (the 7-DoF gauge keeps H singular at mu = 0).  Outputs may be NULL.
 * The parameters are not changed.
 */
mba_status mba_adjoint(mba_problem *problem, const mba_solver_options *opt, double mu, const double *grad_cameras,
                       const double *grad_points, double *grad_obs, double *grad_init_cam, double *grad_init_pt,
                       int32_t *pcg_iters);

/*
 * Cost without any device allocation, for callers that cannot allocate
 * device memory (a framework that owns every allocation through its own pool,
 * a real-time loop where allocating is not allowed, code that must not fail
 * for lack of memory after start-up).  The paper has no counterpart: it is a
 * convenience entry point of this library.
 *
 * All array pointers are DEVICE pointers owned by the caller, in the layouts
 * of mba_problem_create (cameras nc x 9, points np x 3, observations n x 2,
 * cam_idx[n], pt_idx[n]); *d_cost (one double, device memory) receives
 * F = 1/2 sum_k rho(|e_k|^2) in FP64.  Work is enqueued on cuda_stream (NULL =
 * legacy default stream) and the call returns without waiting; the cost is in
 * d_cost when the stream reaches it.  An index out of range yields a NaN cost.
 *
 * Scratch lives in one fixed device array of about 1.8 MB inside the library
 * (every GPU that loads the library holds it until the process exits), so nc
 * may be at most 8192; larger nc returns MBA_ERR_INVALID_ARG, as do NULL
 * pointers, sizes < 1 and a bad loss.  The first call on a device looks up the
 * array's device address (no allocation); make that first call before any
 * stream capture.  Calls share the array: calls whose work overlaps on the GPU
 * race and may return wrong costs, so order them (same stream or events).
 */
mba_status mba_cost_noalloc(const double *d_cameras, int32_t nc, const double *d_points, int32_t np,
                            const double *d_observations, const int32_t *d_cam_idx, const int32_t *d_pt_idx,
                            int64_t n, int32_t loss, double huber_delta, double *d_cost, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Bundle-Adjustment-in-the-Large text files (the problem format of the paper's
 * BAL experiments, Sec. 6): header "nc np n", then n lines "camera point x y",
 * then nc x 9 camera values (angle-axis w, t, f, k1, k2) and np x 3 point
 * values, all whitespace separated.  This is the library's own camera model,
 * so a file's arrays go to mba_problem_create unchanged.  Host only: no GPU.
 *
 * mba_bal_read: parses `path` and returns the sizes; if every array pointer
 * is non-NULL it also fills cameras (nc x 9), points (np x 3), observations
 * (n x 2), cam_idx[n] and pt_idx[n], all owned by the caller (call once with
 * NULL arrays to size them).  Errors: MBA_ERR_INVALID_ARG for an unreadable
 * file, a malformed or truncated file, sizes out of the range
 * mba_problem_create accepts, or an index out of range; MBA_ERR_NONFINITE for
 * a NaN/Inf value.
 * mba_bal_write: writes the same layout, every double with 17 significant
 * digits, so that reading it back returns the same bits.  Errors:
 * MBA_ERR_INVALID_ARG for NULL arguments, sizes < 1 or a failed write.
 * ------------------------------------------------------------------------ */
mba_status mba_bal_read(const char *path, int32_t *nc, int32_t *np, int64_t *n, double *cameras, double *points,
                        double *observations, int32_t *cam_idx, int32_t *pt_idx);
mba_status mba_bal_write(const char *path, int32_t nc, int32_t np, int64_t n, const double *cameras,
                         const double *points, const double *observations, const int32_t *cam_idx,
                         const int32_t *pt_idx);

/* ------------------------------------------------------------------------
 * Batched local bundle adjustment: many small independent problems
 * ("windows", e.g. the sliding windows of a visual SLAM back end) solved in
 * ONE persistent kernel launch, captured once as a CUDA graph.  Each window
 * runs its own Levenberg-Marquardt loop of Alg. 1 (same trust-region rule,
 * Schur elimination of Sec. 3 Eq. 3, PCG of Alg. 2 with the implicit product
 * of Alg. 3, back-substitution of Eq. 4 as mba_solve), with its own radius,
 * accept/reject decisions and stopping test; windows never exchange data.
 * The paper solves one problem at a time; batching is a form of this library.
 *
 * Windows are given concatenated: window w owns cameras
 * [cam_offsets[w], cam_offsets[w+1]), points [pt_offsets[w], pt_offsets[w+1])
 * and observations [obs_offsets[w], obs_offsets[w+1]) of the arrays below
 * (offset arrays have n_windows + 1 entries, start at 0 and never decrease).
 * cam_idx / pt_idx are LOCAL to the window (0 <= cam_idx < the window's
 * camera count).  Limits: 1 <= cameras per window <= 64, every camera and
 * point of a window observed at least once, at most 2^31 - 1 observations in
 * total; otherwise MBA_ERR_INVALID_ARG.  Non-finite inputs give
 * MBA_ERR_NONFINITE.  Precision and loss come from opt (as for
 * mba_problem_create); the FP32-mixed form keeps the PCG dot products, the
 * block inversions and the accept/reject cost in FP64.
 * ------------------------------------------------------------------------ */
typedef struct mba_batch mba_batch;

typedef struct {
    int32_t iterations;        /* LM iterations run, accepted or not */
    int32_t accepted;          /* accepted steps */
    int32_t pcg_iters_total;   /* PCG iterations of the forward solve */
    int32_t status;            /* mba_status of this window */
    double initial_cost;       /* F = 1/2 sum rho(|e|^2) before the first iteration (FP64) */
    double final_cost;
    double final_radius;
    double mu_accepted;        /* mu of the last accepted step; -1 if none */
    int32_t adjoint_pcg_iters; /* PCG iterations of the adjoint solve (0 if none) */
    int32_t pad;
} mba_window_summary;

/* Launch schedule of the batched kernel.  threads_per_cta: 256 or 512;
 * ctas_per_sm: resident windows per SM (1..4, capped by occupancy); schur: how
 * the PCG forms S p (Alg. 3): 1 = implicit (two passes over the observations
 * per iteration), 2 = explicit (S formed once per damped solve as 9x9 blocks,
 * then a dense product per iteration).  Zero fields choose automatically.  The
 * schedule changes the rounding inside a window (results agree to rounding),
 * never the method; a given schedule gives the same bits on every run. */
typedef struct {
    int32_t threads_per_cta;
    int32_t ctas_per_sm;
    int32_t schur;
} mba_batch_schedule;

/* Upstream gradient for the adjoint of every window (same form as
 * mba_adjoint): grad_cameras (total cameras x 9) and grad_points (total
 * points x 3), host arrays in the concatenated order.  With mu < 0 the
 * adjoint of a window uses mu of its last accepted step, and a window without
 * an accepted step (it returned its input unchanged) gets an observation
 * gradient of 0 and the upstream gradient itself as initial-estimate gradient.
 * Windows hold at most 2^24 - 1 points. */
typedef struct {
    const double *grad_cameras;
    const double *grad_points;
    int32_t pcg_max_iter;      /* e.g. 500 */
    int32_t pad;
    double pcg_rel_tol;        /* e.g. 1e-12 */
    double mu;                 /* >= 0: damping of the adjoint system of every window (as the mu
                                  argument of mba_adjoint); < 0: each window's last accepted mu */
} mba_batch_adjoint;

mba_status mba_batch_create(int32_t n_windows, const int64_t *cam_offsets, const int64_t *pt_offsets,
                            const int64_t *obs_offsets, const double *cameras, const double *points,
                            const double *observations, const int32_t *cam_idx, const int32_t *pt_idx,
                            const mba_problem_options *opt, mba_batch **out);
void mba_batch_destroy(mba_batch *batch);
/* Sizes: windows, total cameras / points / observations, largest window camera count. */
mba_status mba_batch_info(const mba_batch *batch, int32_t *n_windows, int64_t *n_cameras, int64_t *n_points,
                          int64_t *n_observations, int32_t *max_window_cameras);
mba_status mba_batch_set_schedule(mba_batch *batch, const mba_batch_schedule *schedule);
mba_status mba_batch_get_schedule(const mba_batch *batch, mba_batch_schedule *schedule);
/* Times each admissible schedule on one solve of this batch (from the current
 * parameters, which are restored afterwards) and keeps the fastest.  The
 * solve options decide the work timed. *ms_best may be NULL. */
mba_status mba_batch_autotune(mba_batch *batch, const mba_solver_options *opt, mba_batch_schedule *chosen,
                              double *ms_best);
/* Solves every window from its current parameters with opt->max_iter LM
 * iterations (opt->function_tol may stop a window early), then, if adj is not
 * NULL, runs each window's adjoint at its solution.  summaries (n_windows
 * entries) and *ms (device time of the launch) may be NULL.  Returns MBA_OK
 * if every window finished with MBA_OK, else the first failing window's
 * status; summaries report every window.  CTAs claim windows longest-first:
 * by an estimate (observations + 10 cameras^2) in a batch's first launch, then by
 * the windows' measured times in the previous launch.  The order changes no
 * result. */
mba_status mba_batch_solve(mba_batch *batch, const mba_solver_options *opt, const mba_batch_adjoint *adj,
                           mba_window_summary *summaries, double *ms);
mba_status mba_batch_get_parameters(const mba_batch *batch, double *cameras, double *points);
/* NULL keeps the current values of that array. */
mba_status mba_batch_set_parameters(mba_batch *batch, const double *cameras, const double *points);
/* Restores the parameters given at creation. */
mba_status mba_batch_reset(mba_batch *batch);
/* Gradients of the last solve with an adjoint: grad_obs (total observations x 2,
 * concatenated input order), grad_init_cam, grad_init_pt.  NULL outputs are skipped. */
mba_status mba_batch_get_gradients(const mba_batch *batch, double *grad_obs, double *grad_init_cam,
                                   double *grad_init_pt);
/* Milliseconds each window's CTA spent on it in the last solve (n_windows entries,
 * input order; %globaltimer on the device).  MBA_ERR_INVALID_ARG before the first solve. */
mba_status mba_batch_window_times(const mba_batch *batch, double *ms);

const char *mba_status_string(mba_status status);
/* Name of the edge type the library's dual-number path evaluates: "BalEdge" (the
 * BAL camera of Sec. 6, Eq. 1's residual), or the user type given at build time
 * (a g2o / Ceres-style user edge, Sec. 5.3).  A library built with a user edge
 * accepts MBA_JACOBIAN_AUTODIFF problems only and no batches. */
const char *mba_edge_name(void);
/* Message describing the last failure on the calling thread ("" if none). */
const char *mba_last_error(void);

/* Process-wide cap on the device memory that one mba_problem_create (its pool
 * plus the set-up scratch it frees before returning) or one mba_batch_create may
 * allocate; 0 (the default) means no cap.  A creation that would exceed the cap
 * returns MBA_ERR_OOM before allocating anything, exactly as if the device had
 * run out of memory, so callers can budget device memory per handle and test
 * their out-of-memory handling without exhausting the GPU.  Handles created
 * earlier are not affected.  The paper has no counterpart (its tables report
 * memory use only).  Always returns MBA_OK. */
mba_status mba_set_device_memory_limit(size_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* MBA_H */
