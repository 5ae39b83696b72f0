// linearize.cu -- residuals, analytic Jacobians and the Hessian blocks
// (Alg. 1: residual/Jacobian step and linear-system step; Sec. 3 Eq. 2).
//
// * camera_table_kernel: per camera, R(w) and the rotation-Jacobian factor M
//   in FP64 (rounded to T for the FP32-mixed form).
// * lin_point_kernel: point-major; per observation e, Jc, Jp and the IRLS
//   weight W, stored sqrt(W)-scaled as structure-of-arrays in point-major order
//   (the layout every later pass streams); per point C = sum Jp~^T Jp~ and
//   w = -sum Jp~^T e~ reduced in shared memory in a fixed order.
// * lin_camera_kernel: camera-major chunks; recomputes Jc (cheaper than
//   re-reading it in another order) and reduces B = sum Jc~^T Jc~ and
//   v = -sum Jc~^T e~ per chunk; cam_finalize sums the chunks of each camera
//   in order.
// * cost kernels: F = 1/2 sum rho(|e|^2) in FP64 for accept/reject.
#include "ff.cuh"
#include "mba_internal.cuh"

namespace mba {

namespace {

inline unsigned grid_for(int64_t n, int per = kBlock) {
    int64_t g = (n + per - 1) / per;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

template <typename T>
__global__ void camera_table_kernel(const double *__restrict__ cams, int32_t nc, T *__restrict__ tab,
                                    double *__restrict__ tab64, float2 *__restrict__ tabff, const DevState *st,
                                    int gate) {
    if (gate == 1 && (st->done || !st->relin)) return;
    if (gate == 2 && st->done) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        double row[kCamTab];
        camera_table_row(cams + 9 * (int64_t)i, row);
        if (tab)
#pragma unroll
            for (int q = 0; q < kCamTab; ++q) tab[(int64_t)i * kCamTab + q] = (T)row[q];
        if (tab64)
#pragma unroll
            for (int q = 0; q < kCamTab; ++q) tab64[(int64_t)i * kCamTab + q] = row[q];
        if (tabff) {  // R, t, f, k1, k2 as float-float
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const ff v = ff_from(row[q]);
                tabff[16 * (int64_t)i + q] = make_float2(v.hi, v.lo);
            }
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const ff v = ff_from(row[18 + q]);
                tabff[16 * (int64_t)i + 9 + q] = make_float2(v.hi, v.lo);
            }
        }
    }
}

__global__ void split_points_kernel(const double *__restrict__ pts, int64_t m, float2 *__restrict__ out,
                                    const DevState *st, int gate) {
    if (gate && st->done) return;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const ff v = ff_from(pts[k]);
        out[k] = make_float2(v.hi, v.lo);
    }
}

// FP32 copy of the pixels for the FP32-mixed linearisation (made once).
__global__ void uv32_kernel(const double2 *__restrict__ uv, int64_t n, float2 *__restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = uv[k];
        out[k] = make_float2((float)v.x, (float)v.y);
    }
}

// FP32 copy of the current points for the FP32-mixed linearisation, one float4
// per point; runs where the linearisation runs (same gate).
__global__ void point_table_kernel(const double *__restrict__ pts, int32_t np, float4 *__restrict__ out,
                                   const DevState *st, int gate) {
    if (gate && (st->done || !st->relin)) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < np; j += gridDim.x * blockDim.x)
        out[j] = make_float4((float)pts[3 * (int64_t)j], (float)pts[3 * (int64_t)j + 1], (float)pts[3 * (int64_t)j + 2],
                             0.f);
}

__global__ void split_uv_kernel(const double2 *__restrict__ uv, int64_t n, float4 *__restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const ff u = ff_from(uv[k].x), v = ff_from(uv[k].y);
        out[k] = make_float4(u.hi, u.lo, v.hi, v.lo);
    }
}

// F = 1/2 sum rho(|e|^2) in float-float (ff.cuh): the BAL projection of each
// observation from the float-float camera table, point and pixel, the loss in
// FP64 where Huber's square root is needed, per-thread sums in float-float.
__global__ void __launch_bounds__(kBlock) cost_partial_ff_kernel(Prob P, double *__restrict__ partial, int gate) {
    __shared__ double sred[kWarps];
    if (gate && P.st->done) return;
    const double d2 = P.delta * P.delta;
    ff acc = ff_from(0.f);
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < P.n; o += (int64_t)gridDim.x * blockDim.x) {
        const int cam = P.pm_cam[o], pt = P.pm_pt[o];
        const float2 *c = P.camff + 16 * (int64_t)cam;
        const float2 *xp = P.ptsff + 3 * (int64_t)pt;
        ff R[9], t[3], X[3];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float2 v = __ldg(c + q);
            R[q] = {v.x, v.y};
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float2 v = __ldg(c + 9 + q), x = __ldg(xp + q);
            t[q] = {v.x, v.y};
            X[q] = {x.x, x.y};
        }
        ff Pc[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            Pc[r] = ff_add(ff_add(ff_mul(R[3 * r], X[0]), ff_mul(R[3 * r + 1], X[1])),
                           ff_add(ff_mul(R[3 * r + 2], X[2]), t[r]));
        const ff iz = ff_rcp(Pc[2]);
        const ff px = ff_neg(ff_mul(Pc[0], iz)), py = ff_neg(ff_mul(Pc[1], iz));
        const float2 fv = __ldg(c + 12), k1v = __ldg(c + 13), k2v = __ldg(c + 14);
        const ff f = {fv.x, fv.y}, k1 = {k1v.x, k1v.y}, k2 = {k2v.x, k2v.y};
        const ff r2 = ff_add(ff_mul(px, px), ff_mul(py, py));
        const ff d = ff_add(ff_from(1.f), ff_mul(r2, ff_add(k1, ff_mul(k2, r2))));
        const ff fd = ff_mul(f, d);
        const float4 uv = __ldg(P.uvff + o);
        const ff e0 = ff_sub(ff_mul(fd, px), ff{uv.x, uv.y});
        const ff e1 = ff_sub(ff_mul(fd, py), ff{uv.z, uv.w});
        const ff sq = ff_add(ff_mul(e0, e0), ff_mul(e1, e1));
        if (P.loss == MBA_LOSS_HUBER && ff_to_double(sq) > d2) {
            const double r = sqrt(ff_to_double(sq));
            acc = ff_add(acc, ff_from(2.0 * P.delta * r - d2));
        } else {
            acc = ff_add(acc, sq);
        }
    }
    const double s = block_sum(ff_to_double(acc), sred);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Per observation of a point-major warp chunk: residual and Jacobians, the
// stored per-observation data, and the nine point-block terms q (packed
// Jp~^T Jp~, then -Jp~^T e~).
template <typename T, bool AD>
__device__ __forceinline__ void lin_point_obs(const Prob &P, int64_t o, int cam, int pt, T *q) {
    constexpr bool FACT = sizeof(T) == 4 && !AD;  // FP32-mixed analytic: no stored Jacobian
    const T *__restrict__ camtab = (const T *)P.camtab;
    T *__restrict__ J = (T *)P.J;
    T *__restrict__ res = (T *)P.res;
    const int64_t np_ = P.npad;
    T X0, X1, X2, u0, u1;
    load_point<T>(P, pt, X0, X1, X2);
    load_uv<T>(P.pm_uv, P.pm_uv32, o, u0, u1);
    T e[2], Jc[18], Jp[6], pz[3];
    edge_eval<T, AD>(camtab + (int64_t)cam * kCamTab, X0, X1, X2, u0, u1, e, Jc, Jp, FACT ? pz : nullptr);
    zero_fixed_columns<T>(P, cam, pt, Jc, Jp);
    T rho, W;
    loss_weight<T>(P.loss, (T)P.delta, e[0] * e[0] + e[1] * e[1], &rho, &W);
    const T sw = sqrt(W);
#pragma unroll
    for (int k = 0; k < 18; ++k) Jc[k] *= sw;
#pragma unroll
    for (int k = 0; k < 6; ++k) Jp[k] *= sw;
    if (FACT) {  // factored form: (px, py, 1/Pz), W Jp and, with a loss, sqrt(W)
#pragma unroll
        for (int k = 0; k < 3; ++k) P.PXpm[k * np_ + o] = (float)pz[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) P.Jph[k * np_ + o] = (float)(sw * Jp[k]);
        if (P.swpm) P.swpm[o] = (float)sw;
    } else {
#pragma unroll
        for (int k = 0; k < 18; ++k) J[k * np_ + o] = Jc[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) J[(18 + k) * np_ + o] = Jp[k];
    }
    e[0] *= sw;
    e[1] *= sw;
    res[o] = e[0];
    res[np_ + o] = e[1];
    q[0] = Jp[0] * Jp[0] + Jp[3] * Jp[3];
    q[1] = Jp[0] * Jp[1] + Jp[3] * Jp[4];
    q[2] = Jp[0] * Jp[2] + Jp[3] * Jp[5];
    q[3] = Jp[1] * Jp[1] + Jp[4] * Jp[4];
    q[4] = Jp[1] * Jp[2] + Jp[4] * Jp[5];
    q[5] = Jp[2] * Jp[2] + Jp[5] * Jp[5];
    q[6] = -(Jp[0] * e[0] + Jp[3] * e[1]);
    q[7] = -(Jp[1] * e[0] + Jp[4] * e[1]);
    q[8] = -(Jp[2] * e[0] + Jp[5] * e[1]);
}

// Point-major linearisation over warp chunks (whole points, <= 32 observations,
// one per lane; or one point with a longer track): every observation's data,
// and per point C = sum Jp~^T Jp~ and w = -sum Jp~^T e~ by a segmented shuffle
// scan in a fixed order, with no shared memory or CTA barrier.
template <typename T, bool AD>
__global__ void __launch_bounds__(kBlock, 4) lin_point_kernel(Prob P, int force) {
    if (!force && (P.st->done || !P.st->relin)) return;
    const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;
    for (int w = blockIdx.x * nwarp + (threadIdx.x >> 5); w < P.n_wchunks; w += gridDim.x * nwarp) {
        const int2 c0 = P.wchunk[w], c1 = P.wchunk[w + 1];
        const int o0 = c0.y, m = c1.y - c0.y;
        T q[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) q[k] = T(0);
        if (m <= 32) {
            const bool act = lane < m;
            const int64_t o = (int64_t)o0 + (act ? lane : 0);
            const int npts = c1.x - c0.x;
            const int rs = lane < npts ? __ldg(P.pt_ptr + c0.x + lane) - o0 : 32;
            const unsigned starts = __reduce_or_sync(full, rs < 32 ? (1u << rs) : 0u);
            const int pt = act ? c0.x + __popc(starts & (0xffffffffu >> (31 - lane))) - 1 : -1 - lane;
            if (act) lin_point_obs<T, AD>(P, o, __ldg(P.pm_cam + o), pt, q);
            // inclusive segmented scan keyed by point; the last lane of each point writes
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int kp = __shfl_up_sync(full, pt, d);
                T v[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = __shfl_up_sync(full, q[k], d);
                if (lane >= d && kp == pt) {
#pragma unroll
                    for (int k = 0; k < 9; ++k) q[k] += v[k];
                }
            }
            const int nxt = __shfl_down_sync(full, pt, 1);
            if (act && (lane == m - 1 || nxt != pt)) {
#pragma unroll
                for (int k = 0; k < 6; ++k) P.Hll[6 * (int64_t)pt + k] = (double)q[k];
#pragma unroll
                for (int k = 0; k < 3; ++k) P.w[3 * (int64_t)pt + k] = (double)q[6 + k];
            }
        } else {
            // one point with a long track: 32-observation slices, then a tree
            const int pt = c0.x;
            for (int base = 0; base < m; base += 32) {
                if (base + lane < m) {
                    const int64_t o = (int64_t)o0 + base + lane;
                    T qq[9];
                    lin_point_obs<T, AD>(P, o, __ldg(P.pm_cam + o), pt, qq);
#pragma unroll
                    for (int k = 0; k < 9; ++k) q[k] += qq[k];
                }
            }
#pragma unroll
            for (int k = 0; k < 9; ++k)
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) q[k] += __shfl_xor_sync(full, q[k], d);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) P.Hll[6 * (int64_t)pt + k] = (double)q[k];
#pragma unroll
                for (int k = 0; k < 3; ++k) P.w[3 * (int64_t)pt + k] = (double)q[6 + k];
            }
        }
    }
}

// One warp per camera chunk: each lane accumulates the 54 block terms of its
// observations, then one shuffle tree per chunk (a CTA-wide reduction per
// chunk of a few hundred observations cost as much as the Jacobians).
// The FP32 instance is held to two CTAs per SM (128 registers); the FP64 one is
// bound by the FP64 pipe and keeps its registers.
template <typename T, bool AD>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 2 : 1) lin_camera_kernel(Prob P, int force) {
    if (!force && (P.st->done || !P.st->relin)) return;
    __shared__ T ctabs[kWarps][kCamTab];
    const T *__restrict__ camtab = (const T *)P.camtab;
    const T delta = (T)P.delta;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *ctab = ctabs[wid];
    for (int c = blockIdx.x * kWarps + wid; c < P.n_cchunks; c += gridDim.x * kWarps) {
        const int cam = P.cchunk_cam[c];
        const int b0 = P.cchunk_beg[c], b1 = P.cchunk_beg[c + 1];
        __syncwarp();
        if (lane < kCamTab) ctab[lane] = camtab[(int64_t)cam * kCamTab + lane];
        __syncwarp();
        T acc[54];
#pragma unroll
        for (int q = 0; q < 54; ++q) acc[q] = T(0);
        // two-deep pipeline over this lane's observations (the point index two
        // ahead, the point and pixels one ahead), so that the dependent point
        // gather is in flight while the previous observation is worked
        int s = b0 + lane;
        int pa = s < b1 ? P.cm_pt[s] : 0;
        int pb = s + 32 < b1 ? P.cm_pt[s + 32] : 0;
        T Xa0 = T(0), Xa1 = T(0), Xa2 = T(0), ua0 = T(0), ua1 = T(0);
        if (s < b1) {
            load_point<T>(P, pa, Xa0, Xa1, Xa2);
            load_uv<T>(P.cm_uv, P.cm_uv32, s, ua0, ua1);
        }
        for (; s < b1; s += 32) {
            const int pt = pa;
            const T X0 = Xa0, X1 = Xa1, X2 = Xa2, u0 = ua0, u1 = ua1;
            const int pc = s + 64 < b1 ? P.cm_pt[s + 64] : 0;
            if (s + 32 < b1) {
                load_point<T>(P, pb, Xa0, Xa1, Xa2);
                load_uv<T>(P.cm_uv, P.cm_uv32, s + 32, ua0, ua1);
            }
            pa = pb;
            pb = pc;
            T e[2], Jc[18], Jp[6], pz[3];
            edge_eval<T, AD, true, false>(ctab, X0, X1, X2, u0, u1, e, Jc, Jp, (sizeof(T) == 4 && !AD) ? pz : nullptr);
            zero_fixed_columns<T>(P, cam, pt, Jc, (T *)nullptr);
            T rho, W;
            loss_weight<T>(P.loss, delta, e[0] * e[0] + e[1] * e[1], &rho, &W);
            const T sw = sqrt(W);
#pragma unroll
            for (int q = 0; q < 18; ++q) Jc[q] *= sw;
            e[0] *= sw;
            e[1] *= sw;
            // what the PCG camera pass reads in camera-major order: the stored
            // Jacobian (FP64, or any dual-number Jacobian), else the factored
            // form's (R X, 1/Pz)
            if ((sizeof(T) == 8 || AD) && P.JcmT) {
#pragma unroll
                for (int q = 0; q < 18; ++q) ((T *)P.JcmT)[(int64_t)q * P.npad + s] = Jc[q];
            }
            if (sizeof(T) == 4 && !AD && P.fact) {
                ((float4 *)P.RXcm)[s] = make_float4((float)(ctab[0] * X0 + ctab[1] * X1 + ctab[2] * X2),
                                                    (float)(ctab[3] * X0 + ctab[4] * X1 + ctab[5] * X2),
                                                    (float)(ctab[6] * X0 + ctab[7] * X1 + ctab[8] * X2), (float)pz[2]);
            }
            int idx = 0;
#pragma unroll
            for (int a = 0; a < 9; ++a)
#pragma unroll
                for (int b = a; b < 9; ++b) acc[idx++] += Jc[a] * Jc[b] + Jc[9 + a] * Jc[9 + b];
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[45 + a] -= Jc[a] * e[0] + Jc[9 + a] * e[1];
        }
        // lane q (and q - 32) ends with sum q
        double mine0 = 0.0, mine1 = 0.0;
#pragma unroll
        for (int q = 0; q < 54; ++q) {
            T v = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == (q & 31)) {
                if (q < 32) mine0 = (double)v;
                else mine1 = (double)v;
            }
        }
        P.cpart[54 * (int64_t)c + lane] = mine0;
        if (lane < 22) P.cpart[54 * (int64_t)c + 32 + lane] = mine1;
    }
}

__global__ void cam_finalize_kernel(Prob P, const int32_t *__restrict__ cfirst, int force) {
    if (!force && (P.st->done || !P.st->relin)) return;
    const int64_t total = (int64_t)P.nc * 54;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / 54), q = (int)(t % 54);
        double s = 0.0;
        for (int c = cfirst[i]; c < cfirst[i + 1]; ++c) s += P.cpart[54 * (int64_t)c + q];
        if (q < 45) P.Hpp[45 * (int64_t)i + q] = s;
        else P.v[9 * (int64_t)i + (q - 45)] = s;
    }
}

// FP64 cost over the point-major observations; fixed grid and order.
template <bool AD>
__global__ void __launch_bounds__(kBlock) cost_partial_kernel(Prob P, const double *__restrict__ pts,
                                                               double *__restrict__ partial, int gate) {
    __shared__ double sred[kWarps];
    if (gate && P.st->done) return;
    double acc = 0.0;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < P.n; o += (int64_t)gridDim.x * blockDim.x) {
        const int cam = P.pm_cam[o], pt = P.pm_pt[o];
        const double2 uv = P.pm_uv[o];
        double e[2];
        edge_residual<double, AD>(P.camtab64 + (int64_t)cam * kCamTab, pts[3 * (int64_t)pt],
                                  pts[3 * (int64_t)pt + 1], pts[3 * (int64_t)pt + 2], uv.x, uv.y, e);
        double rho, W;
        loss_weight<double>(P.loss, P.delta, e[0] * e[0] + e[1] * e[1], &rho, &W);
        acc += rho;
    }
    const double s = block_sum(acc, sred);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void cost_final_kernel(const double *__restrict__ partial, int nb, double *out, double *out2,
                                  const DevState *st, int gate) {
    __shared__ double sred[kWarps];
    if (gate && st->done) return;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    const double s = block_sum(acc, sred);
    if (threadIdx.x == 0) {
        *out = 0.5 * s;
        if (out2) *out2 = 0.5 * s;
    }
}

template <typename T, bool AD>
__global__ void __launch_bounds__(kBlock) evaluate_slice_kernel(Prob P, const int32_t *__restrict__ ci,
                                                                 const int32_t *__restrict__ pi,
                                                                 const double2 *__restrict__ uvs, int64_t m,
                                                                 double *__restrict__ eo, double *__restrict__ jco,
                                                                 double *__restrict__ jpo) {
    const T *__restrict__ camtab = (const T *)P.camtab;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int cam = ci[k], pt = pi[k];
        const double2 uv = uvs[k];
        T e[2], Jc[18], Jp[6];
        edge_eval<T, AD>(camtab + (int64_t)cam * kCamTab, (T)P.pts[3 * (int64_t)pt], (T)P.pts[3 * (int64_t)pt + 1],
                         (T)P.pts[3 * (int64_t)pt + 2], (T)uv.x, (T)uv.y, e, Jc, Jp);
        eo[2 * k] = (double)e[0];
        eo[2 * k + 1] = (double)e[1];
#pragma unroll
        for (int q = 0; q < 18; ++q) jco[18 * k + q] = (double)Jc[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) jpo[6 * k + q] = (double)Jp[q];
    }
}

}  // namespace

int cost_grid(const Prob &P) { return (int)grid_for(P.n); }

cudaError_t launch_camera_tables(const Prob &P, const double *cams, bool for_lin, cudaStream_t s) {
    const unsigned g = grid_for(P.nc, 128);
    if (for_lin) {
        if (P.fp32)
            camera_table_kernel<float><<<g, 128, 0, s>>>(cams, P.nc, (float *)P.camtab, nullptr, nullptr, P.st, 1);
        else
            camera_table_kernel<double><<<g, 128, 0, s>>>(cams, P.nc, (double *)P.camtab, nullptr, nullptr, P.st, 1);
    } else {
        camera_table_kernel<double><<<g, 128, 0, s>>>(cams, P.nc, nullptr, P.camtab64, P.camff, P.st, 2);
    }
    return cudaGetLastError();
}

cudaError_t launch_camera_tables_forced(const Prob &P, const double *cams, cudaStream_t s) {
    const unsigned g = grid_for(P.nc, 128);
    if (P.fp32)
        camera_table_kernel<float><<<g, 128, 0, s>>>(cams, P.nc, (float *)P.camtab, P.camtab64, P.camff, P.st, 0);
    else
        camera_table_kernel<double><<<g, 128, 0, s>>>(cams, P.nc, (double *)P.camtab, P.camtab64, nullptr, P.st, 0);
    return cudaGetLastError();
}

cudaError_t launch_split_observations(const Prob &P, cudaStream_t s) {
    if (P.uvff) split_uv_kernel<<<grid_for(P.n), kBlock, 0, s>>>(P.pm_uv, P.n, P.uvff);
    if (P.pm_uv32) uv32_kernel<<<grid_for(P.n), kBlock, 0, s>>>(P.pm_uv, P.n, P.pm_uv32);
    if (P.cm_uv32) uv32_kernel<<<grid_for(P.n), kBlock, 0, s>>>(P.cm_uv, P.n, P.cm_uv32);
    return cudaGetLastError();
}

template <typename T, bool AD>
static void launch_lin_pair(const Prob &P, int force, cudaStream_t s) {
    int nbp = (P.n_wchunks + kWarps - 1) / kWarps;
    if (nbp > 152 * 16) nbp = 152 * 16;
    lin_point_kernel<T, AD><<<nbp < 1 ? 1 : nbp, kBlock, 0, s>>>(P, force);
    int nbc = (P.n_cchunks + kWarps - 1) / kWarps;
    if (nbc > 152 * 16) nbc = 152 * 16;
    lin_camera_kernel<T, AD><<<nbc < 1 ? 1 : nbc, kBlock, 0, s>>>(P, force);
}

cudaError_t launch_linearize_impl(const Prob &P, const int32_t *cfirst, int force, cudaStream_t s) {
    if (P.fp32) {
        point_table_kernel<<<grid_for(P.np), kBlock, 0, s>>>(P.pts, P.np, P.pts32, P.st, force ? 0 : 1);
        if (P.autodiff) launch_lin_pair<float, true>(P, force, s);
        else launch_lin_pair<float, false>(P, force, s);
    } else {
        if (P.autodiff) launch_lin_pair<double, true>(P, force, s);
        else launch_lin_pair<double, false>(P, force, s);
    }
    cam_finalize_kernel<<<grid_for((int64_t)P.nc * 54), kBlock, 0, s>>>(P, cfirst, force);
    return cudaGetLastError();
}

cudaError_t launch_cost_impl(const Prob &P, const double *pts, double *partial, double *out, double *out2, int gate,
                             cudaStream_t s, bool ff) {
    const int nb = cost_grid(P);
    if (ff && P.camff && P.uvff && P.ptsff) {
        split_points_kernel<<<grid_for(3 * (int64_t)P.np), kBlock, 0, s>>>(pts, 3 * (int64_t)P.np, P.ptsff, P.st, gate);
        cost_partial_ff_kernel<<<nb, kBlock, 0, s>>>(P, partial, gate);
        cost_final_kernel<<<1, kBlock, 0, s>>>(partial, nb, out, out2, P.st, gate);
        return cudaGetLastError();
    }
    if (P.autodiff) cost_partial_kernel<true><<<nb, kBlock, 0, s>>>(P, pts, partial, gate);
    else cost_partial_kernel<false><<<nb, kBlock, 0, s>>>(P, pts, partial, gate);
    cost_final_kernel<<<1, kBlock, 0, s>>>(partial, nb, out, out2, P.st, gate);
    return cudaGetLastError();
}

cudaError_t launch_evaluate_slice(const Prob &P, const int32_t *ci, const int32_t *pi, const double2 *uv, int64_t m,
                                  double *e, double *jc, double *jp, cudaStream_t s) {
    const unsigned g = grid_for(m);
    if (P.fp32) {
        if (P.autodiff) evaluate_slice_kernel<float, true><<<g, kBlock, 0, s>>>(P, ci, pi, uv, m, e, jc, jp);
        else evaluate_slice_kernel<float, false><<<g, kBlock, 0, s>>>(P, ci, pi, uv, m, e, jc, jp);
    } else {
        if (P.autodiff) evaluate_slice_kernel<double, true><<<g, kBlock, 0, s>>>(P, ci, pi, uv, m, e, jc, jp);
        else evaluate_slice_kernel<double, false><<<g, kBlock, 0, s>>>(P, ci, pi, uv, m, e, jc, jp);
    }
    return cudaGetLastError();
}

}  // namespace mba
