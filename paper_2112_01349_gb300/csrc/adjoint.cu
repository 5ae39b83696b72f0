// adjoint.cu -- gradient of the solved state for the differentiable BA layer
// (the paper has no counterpart; it reuses the Schur-PCG of Alg. 2/3).
//
// At the solution x* with M = H(x*) + mu D, the implicit function theorem on
// the optimality condition J^T W e = 0 (e = pi(x) - u) gives d(x*)/du_k =
// M^-1 J_k^T W_k.  For an upstream gradient gbar = dL/dx*, v = M^-1 gbar is
// found by the same Schur elimination, PCG and back-substitution as an LM
// step (right-hand side gbar in place of the gradient), and then
//   dL/du_k = W_k J_k v              (adjoint_obs_kernel, per observation)
//   dL/dx0  = mu D v                 (adjoint_init_kernel: the last LM step is
//                                      the proximal step around the previous
//                                      iterate, damped by mu D)
#include "mba_internal.cuh"

namespace mba {

namespace {

__device__ __forceinline__ double damp_diag(int damping, double d) {
    if (damping == MBA_DAMP_IDENTITY) return 1.0;
    return fmin(fmax(d, 1e-6), 1e32);
}

// dL/du_k = W_k (Jc_k v_c + Jp_k v_p) for a slice of observations in the
// caller's order; the Jacobian and W are recomputed at x* in the problem's
// precision, the product is accumulated in FP64.
template <typename T, bool AD>
__global__ void __launch_bounds__(kBlock) adjoint_obs_kernel(Prob P, const int32_t *__restrict__ ci,
                                                              const int32_t *__restrict__ pi,
                                                              const double2 *__restrict__ uvs, int64_t m,
                                                              double *__restrict__ out) {
    const T *__restrict__ camtab = (const T *)P.camtab;
    const T delta = (T)P.delta;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int cam = ci[k], pt = pi[k];
        const double2 uv = uvs[k];
        T e[2], Jc[18], Jp[6];
        edge_eval<T, AD>(camtab + (int64_t)cam * kCamTab, (T)P.pts[3 * (int64_t)pt], (T)P.pts[3 * (int64_t)pt + 1],
                         (T)P.pts[3 * (int64_t)pt + 2], (T)uv.x, (T)uv.y, e, Jc, Jp);
        zero_fixed_columns<T>(P, cam, pt, Jc, Jp);
        T rho, W;
        loss_weight<T>(P.loss, delta, e[0] * e[0] + e[1] * e[1], &rho, &W);
        const double *vc = P.x + (int64_t)cam * kVec;
        const double *vp = P.dp + 3 * (int64_t)pt;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < 9; ++a) s = fma((double)Jc[r * 9 + a], vc[a], s);
#pragma unroll
            for (int a = 0; a < 3; ++a) s = fma((double)Jp[r * 3 + a], vp[a], s);
            out[2 * k + r] = (double)W * s;
        }
    }
}

// dL/dx0 = mu D v, D = clamp(diag(B, C), 1e-6, 1e32) (or I), into cams_new / pts_new
__global__ void adjoint_init_kernel(Prob P, int damping, double mu) {
    const int64_t ncv = 9 * (int64_t)P.nc, total = ncv + 3 * (int64_t)P.np;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < ncv) {
            const int64_t i = t / 9, a = t % 9;
            const double d = damp_diag(damping, P.Hpp[45 * i + sym9((int)a, (int)a)]);
            P.cams_new[t] = mu * d * P.x[i * kVec + a];
        } else {
            const int64_t u = t - ncv, j = u / 3, a = u % 3;
            const double d = damp_diag(damping, P.Hll[6 * j + sym3((int)a, (int)a)]);
            P.pts_new[u] = mu * d * P.dp[u];
        }
    }
}

}  // namespace

cudaError_t launch_adjoint_obs(const Prob &P, const int32_t *ci, const int32_t *pi, const double2 *uv, int64_t m,
                               double *out, cudaStream_t s) {
    int64_t g = (m + kBlock - 1) / kBlock;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    const unsigned gu = (unsigned)g;
    if (P.fp32) {
        if (P.autodiff) adjoint_obs_kernel<float, true><<<gu, kBlock, 0, s>>>(P, ci, pi, uv, m, out);
        else adjoint_obs_kernel<float, false><<<gu, kBlock, 0, s>>>(P, ci, pi, uv, m, out);
    } else {
        if (P.autodiff) adjoint_obs_kernel<double, true><<<gu, kBlock, 0, s>>>(P, ci, pi, uv, m, out);
        else adjoint_obs_kernel<double, false><<<gu, kBlock, 0, s>>>(P, ci, pi, uv, m, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_init(const Prob &P, int damping, double mu, cudaStream_t s) {
    const int64_t total = 9 * (int64_t)P.nc + 3 * (int64_t)P.np;
    int64_t g = (total + kBlock - 1) / kBlock;
    if (g > 152 * 16) g = 152 * 16;
    adjoint_init_kernel<<<(unsigned)g, kBlock, 0, s>>>(P, damping, mu);
    return cudaGetLastError();
}

}  // namespace mba
