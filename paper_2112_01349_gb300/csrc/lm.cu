// lm.cu -- device-side Levenberg-Marquardt control (Alg. 1 outer loop with the
// Ceres-style trust region the supplement names).  Every decision is taken on
// the device so a whole solve is issued without a host round trip.
//
// Rules: mu = 1 / radius; gain = (F - F') / model_decrease; a step is accepted
// iff model_decrease > 0, F' is finite and gain > min_relative_decrease.
// Accepted: radius /= max(1/3, 1 - (2 gain - 1)^3), decrease factor = 2.
// Rejected: radius /= factor, factor *= 2.  radius stays in [1e-32, 1e16].
// A rejected iteration counts and keeps the linearisation.  An iteration whose
// damped blocks are not all positive definite (no step) is rejected.
#include "mba_internal.cuh"

namespace mba {

namespace {

__global__ void state_init_kernel(DevState *st, double radius, double mu_override, int keep_cost) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double cost = st->cost;
    DevState z = {};
    z.radius = radius;
    z.factor = 2.0;
    z.mu = mu_override >= 0.0 ? mu_override : 1.0 / radius;
    z.mu_override = mu_override;
    z.relin = 1;
    if (keep_cost) z.cost = cost;
    *st = z;
}

__global__ void lm_update_kernel(DevState *st, mba_iteration *trace, int trace_cap, double min_rel_dec,
                                 double function_tol) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (st->done) {
        st->accepted = 0;
        return;
    }
    if (st->err != 0) {
        st->done = 1;
        st->accepted = 0;
        return;
    }
    // a damped block that was not positive definite: no step this iteration,
    // which counts as rejected (mu grows, the linearisation is kept)
    const int blockfail = st->blockfail;
    if (blockfail) {
        st->cost_new = nan("");
        st->model_dec = 0.0;
        st->pcg_iters = 0;
        st->pcg_rel_res = 0.0;
        st->blockfail = 0;
    }
    const double F = st->cost, Fn = st->cost_new, L = st->model_dec;
    const double gain = blockfail ? nan("") : (F - Fn) / L;
    const int accept = !blockfail && (L > 0.0) && isfinite(Fn) && (gain > min_rel_dec);
    const int it = st->iter;
    if (trace && it < trace_cap) {
        mba_iteration t;
        t.cost = F;
        t.cost_new = Fn;
        t.model_decrease = L;
        t.mu = st->mu;
        t.gain = gain;
        t.accepted = accept;
        t.pcg_iters = st->pcg_iters;
        t.pcg_rel_residual = st->pcg_rel_res;
        trace[it] = t;
    }
    double radius = st->radius;
    if (accept) {
        const double t = 2.0 * gain - 1.0;
        const double shrink = 1.0 - t * t * t;
        radius = radius / fmax(shrink, 1.0 / 3.0);
        st->factor = 2.0;
        if (function_tol > 0.0 && fabs(F - Fn) < function_tol * F) st->done = 1;
        st->cost = Fn;
        st->mu_accepted = st->mu;
        st->accepted_total += 1;
    } else {
        radius = radius / st->factor;
        st->factor *= 2.0;
    }
    st->radius = fmin(fmax(radius, 1e-32), 1e16);
    st->gain = gain;
    st->accepted = accept;
    st->relin = accept;
    st->pcg_total += st->pcg_iters;
    st->iter = it + 1;
}

__global__ void accept_copy_kernel(double *cams, const double *cams_new, int64_t ncv, double *pts,
                                   const double *pts_new, int64_t npv, const DevState *st) {
    if (!st->accepted) return;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncv + npv; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < ncv) cams[t] = cams_new[t];
        else pts[t - ncv] = pts_new[t - ncv];
    }
}

}  // namespace

cudaError_t launch_state_init(const Prob &P, double radius, double mu_override, int keep_cost, cudaStream_t s) {
    state_init_kernel<<<1, 32, 0, s>>>(P.st, radius, mu_override, keep_cost);
    return cudaGetLastError();
}

cudaError_t launch_lm_update(const Prob &P, const mba_solver_options &o, cudaStream_t s) {
    lm_update_kernel<<<1, 32, 0, s>>>(P.st, P.trace, P.trace_cap, o.min_relative_decrease, o.function_tol);
    return cudaGetLastError();
}

cudaError_t launch_accept(const Prob &P, cudaStream_t s) {
    const int64_t tot = 9 * (int64_t)P.nc + 3 * (int64_t)P.np;
    int64_t g = (tot + kBlock - 1) / kBlock;
    if (g > 152 * 8) g = 152 * 8;
    accept_copy_kernel<<<(unsigned)g, kBlock, 0, s>>>(P.cams, P.cams_new, 9 * (int64_t)P.nc, P.pts, P.pts_new,
                                                      3 * (int64_t)P.np, P.st);
    return cudaGetLastError();
}

}  // namespace mba
