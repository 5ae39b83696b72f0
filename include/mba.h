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

typedef struct {
    int32_t precision;   /* mba_precision.  FP32_MIXED: Jacobian, Hessian blocks and the
                            PCG Schur product in FP32; block inversions, PCG dot
                            products and norms, cost and accept/reject in FP64. */
    int32_t loss;        /* mba_loss; cost F = 1/2 sum rho(|e|^2) (Eq. 1 with Sigma = I) */
    double huber_delta;  /* Huber threshold in pixels (MBA_LOSS_HUBER) */
    void *cuda_stream;   /* cudaStream_t to run on; NULL = the legacy default stream */
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
 * pcg_rel_tol 1e-10, DIAG damping, radius 1e4, min decrease 1e-3, function_tol 0. */
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

const char *mba_status_string(mba_status status);
/* Message describing the last failure on the calling thread ("" if none). */
const char *mba_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MBA_H */
