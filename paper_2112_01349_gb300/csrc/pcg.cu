// pcg.cu -- damping and block inversions, the persistent PCG on the reduced
// camera system (Alg. 2) with the implicit Schur product (Alg. 3), and the
// point back-substitution (Sec. 3 Eq. 4) with the linear model decrease.
//
// Implicit product S p = B~ p - E C~^-1 E^T p, one pass over the point-major
// observation stream per PCG iteration:
//   per observation  t_k = Jc~_k p_i(k),  u_k = Jp~_k^T t_k        (E^T p)
//   per point        b_j = C~_j^-1 sum_k u_k                       (C~^-1)
//   per observation  y_k = Jc~_k^T (Jp~_k b_j) added into camera i(k) (E b)
// so the 24 Jacobian values of each observation are read once per iteration.
// The camera-side work (B~ p, the preconditioner B~^-1 r, dot products,
// axpys) is FP64 in both precisions, spread over all CTAs, three cameras per
// warp, with bounded grid barriers between the phases.
#include "mba_internal.cuh"

namespace mba {

namespace {

// ---------------------------------------------------------------------------
// damping: B~ = B + mu D_B, C~ = C + mu D_C (D = clamp(diag, 1e-6, 1e32), or I)
// B~ is stored full, with its inverse (Cholesky, FP64) as the block-Jacobi
// preconditioner; C~^-1 (adjugate, FP64) is stored packed in T.  A block that
// is not positive definite sets DevState::blockfail: the LM loop rejects the
// iteration (mu grows), single-step entry points report MBA_ERR_NONFINITE.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double damp_term(int damping, double d) {
    if (damping == MBA_DAMP_IDENTITY) return 1.0;
    return fmin(fmax(d, 1e-6), 1e32);
}

__device__ __forceinline__ double current_mu(const DevState *st) {
    return st->mu_override >= 0.0 ? st->mu_override : 1.0 / st->radius;
}

// Warp-collective inverse of a symmetric positive definite 9x9 matrix in FP64.
// A (shared memory, 81 doubles, both triangles set) is overwritten by its
// lower Cholesky factor (right-looking: lane-parallel column scaling and
// trailing update), Y (shared, 81) receives L^-1 by forward substitution, one
// column per lane, and inv (global, row-major) = L^-T L^-1.  Returns false on
// every lane, writing nothing, if a pivot is not positive.  The chains are
// short (about 9 steps per column) where one thread per matrix would run
// hundreds of dependent FP64 operations.
__device__ bool warp_spd_inverse9(double *A, double *Y, double *il, double *inv) {
    const int lane = threadIdx.x & 31;
    // this lane's lower-triangle entries (r >= c) of the trailing updates
    int e_r[2], e_c[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int e = lane + 32 * h;
        int r = 0;
        while (r < 9 && (r + 1) * (r + 2) / 2 <= e) ++r;
        e_r[h] = r;
        e_c[h] = e - r * (r + 1) / 2;
    }
    for (int j = 0; j < 9; ++j) {
        __syncwarp();
        const double d = A[j * 9 + j];
        if (!(d > 0.0) || !isfinite(d)) return false;
        const double l = sqrt(d), ilj = 1.0 / l;
        __syncwarp();
        if (lane == 0) {
            A[j * 9 + j] = l;
            il[j] = ilj;
        }
        if (lane > j && lane < 9) A[lane * 9 + j] *= ilj;
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = e_r[h], c = e_c[h];
            if (lane + 32 * h < 45 && c > j) A[r * 9 + c] -= A[r * 9 + j] * A[c * 9 + j];
        }
    }
    __syncwarp();
    if (lane < 9) {  // column `lane` of L^-1 (rows >= lane)
        const int c = lane;
        for (int r = 0; r < 9; ++r) {
            if (r < c) {
                Y[r * 9 + c] = 0.0;
                continue;
            }
            double s = r == c ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) s -= A[r * 9 + k] * Y[k * 9 + c];
            Y[r * 9 + c] = s * il[r];
        }
    }
    __syncwarp();
    for (int e = lane; e < 81; e += 32) {
        const int r = e / 9, c = e - 9 * (e / 9), k0 = r > c ? r : c;
        double s = 0.0;
        for (int k = k0; k < 9; ++k) s += Y[k * 9 + r] * Y[k * 9 + c];
        inv[e] = s;
    }
    return true;
}

// One warp per camera: B~ (full, stored for the PCG's B~ p) and its inverse.
constexpr int kDampWarps = 4;
__global__ void __launch_bounds__(32 * kDampWarps) damp_cameras_kernel(Prob P, int damping) {
    __shared__ double sA[kDampWarps][81], sY[kDampWarps][81], sil[kDampWarps][9];
    DevState *st = P.st;
    if (st->done) return;
    const double mu = current_mu(st);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->mu = mu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = blockIdx.x * kDampWarps + wid; i < P.nc; i += gridDim.x * kDampWarps) {
        double *A = sA[wid];
        __syncwarp();
        for (int e = lane; e < 81; e += 32) {
            const int a = e / 9, b = e - 9 * (e / 9);
            double v = P.Hpp[45 * (int64_t)i + sym9(a, b)];
            if (a == b) v += mu * damp_term(damping, v);
            A[e] = v;
            P.Bd[81 * (int64_t)i + e] = v;
        }
        __syncwarp();
        if (!warp_spd_inverse9(A, sY[wid], sil[wid], P.Binv + 81 * (int64_t)i) && lane == 0)
            atomicExch(&st->blockfail, 1);
    }
}

template <typename T>
__global__ void damp_points_kernel(Prob P, int damping) {
    DevState *st = P.st;
    if (st->done) return;
    const double mu = current_mu(st);
    T *Ci = (T *)P.Cinv;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.np; j += (int64_t)gridDim.x * blockDim.x) {
        const double *h = P.Hll + 6 * j;
        const double a00 = h[0] + mu * damp_term(damping, h[0]), a01 = h[1], a02 = h[2];
        const double a11 = h[3] + mu * damp_term(damping, h[3]), a12 = h[4];
        const double a22 = h[5] + mu * damp_term(damping, h[5]);
        const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
        const double det = a00 * c00 + a01 * c01 + a02 * c02;
        if (!(det > 0.0) || !isfinite(det)) {
            atomicExch(&st->blockfail, 1);
            continue;
        }
        const double id = 1.0 / det;
        Ci[6 * j + 0] = (T)(c00 * id);
        Ci[6 * j + 1] = (T)(c01 * id);
        Ci[6 * j + 2] = (T)(c02 * id);
        Ci[6 * j + 3] = (T)((a00 * a22 - a02 * a02) * id);
        Ci[6 * j + 4] = (T)((a02 * a01 - a00 * a12) * id);
        Ci[6 * j + 5] = (T)((a00 * a11 - a01 * a01) * id);
    }
}

// ---------------------------------------------------------------------------
// Schur-Jacobi preconditioner (solver variant): S~_ii = B~_i - sum_k
// Jc~_k^T G_k Jc~_k over the observations k of camera i, G_k = Jp~_k C~_j^-1
// Jp~_k^T (2x2).  Camera-major chunks recompute the Jacobian (as the
// linearisation's camera pass does) and write 45 packed chunk sums; each
// camera then subtracts its chunk sums from B~_i in chunk order and, if the
// result is positive definite, replaces the preconditioner block by its
// inverse (Cholesky, FP64).  Otherwise B~_i^-1 stays.
// ---------------------------------------------------------------------------
template <typename T, bool AD>
__global__ void __launch_bounds__(kBlock) sj_camera_kernel(Prob P) {
    if (P.st->done) return;
    __shared__ T ctab[kCamTab];
    __shared__ double red[kWarps][45];
    const T *__restrict__ camtab = (const T *)P.camtab;
    const T *__restrict__ Ci = (const T *)P.Cinv;
    const T delta = (T)P.delta;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = blockIdx.x; c < P.n_cchunks; c += gridDim.x) {
        const int cam = P.cchunk_cam[c];
        const int b0 = P.cchunk_beg[c], b1 = P.cchunk_beg[c + 1];
        __syncthreads();
        if (threadIdx.x < kCamTab) ctab[threadIdx.x] = camtab[(int64_t)cam * kCamTab + threadIdx.x];
        __syncthreads();
        T acc[45];
#pragma unroll
        for (int q = 0; q < 45; ++q) acc[q] = T(0);
        for (int s = b0 + threadIdx.x; s < b1; s += kBlock) {
            const int pt = P.cm_pt[s];
            T X0, X1, X2, u0, u1;
            load_point<T>(P, pt, X0, X1, X2);
            load_uv<T>(P.cm_uv, P.cm_uv32, s, u0, u1);
            T e[2], Jc[18], Jp[6];
            edge_eval<T, AD>(ctab, X0, X1, X2, u0, u1, e, Jc, Jp);
            zero_fixed_columns<T>(P, cam, pt, Jc, Jp);
            T rho, W;
            loss_weight<T>(P.loss, delta, e[0] * e[0] + e[1] * e[1], &rho, &W);
            T c6[6], q0[3], q1[3];
#pragma unroll
            for (int q = 0; q < 6; ++q) c6[q] = Ci[6 * (int64_t)pt + q];
            // Q = Jp C~^-1 (rows), G = W^2 Q Jp^T
            q0[0] = c6[0] * Jp[0] + c6[1] * Jp[1] + c6[2] * Jp[2];
            q0[1] = c6[1] * Jp[0] + c6[3] * Jp[1] + c6[4] * Jp[2];
            q0[2] = c6[2] * Jp[0] + c6[4] * Jp[1] + c6[5] * Jp[2];
            q1[0] = c6[0] * Jp[3] + c6[1] * Jp[4] + c6[2] * Jp[5];
            q1[1] = c6[1] * Jp[3] + c6[3] * Jp[4] + c6[4] * Jp[5];
            q1[2] = c6[2] * Jp[3] + c6[4] * Jp[4] + c6[5] * Jp[5];
            const T w2 = W * W;
            const T g00 = w2 * (q0[0] * Jp[0] + q0[1] * Jp[1] + q0[2] * Jp[2]);
            const T g01 = w2 * (q0[0] * Jp[3] + q0[1] * Jp[4] + q0[2] * Jp[5]);
            const T g11 = w2 * (q1[0] * Jp[3] + q1[1] * Jp[4] + q1[2] * Jp[5]);
            T F0[9], F1[9];
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                F0[b] = g00 * Jc[b] + g01 * Jc[9 + b];
                F1[b] = g01 * Jc[b] + g11 * Jc[9 + b];
            }
            int idx = 0;
#pragma unroll
            for (int a = 0; a < 9; ++a)
#pragma unroll
                for (int b = a; b < 9; ++b) acc[idx++] += Jc[a] * F0[b] + Jc[9 + a] * F1[b];
        }
#pragma unroll
        for (int q = 0; q < 45; ++q) {
            T v = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[wid][q] = (double)v;
        }
        __syncthreads();
        if (threadIdx.x < 45) {
            double s = 0.0;
            for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
            P.cpart[54 * (int64_t)c + threadIdx.x] = s;
        }
    }
}

__global__ void __launch_bounds__(32 * kDampWarps) sj_finalize_kernel(Prob P, const int32_t *__restrict__ cfirst) {
    __shared__ double sA[kDampWarps][81], sY[kDampWarps][81], sil[kDampWarps][9];
    if (P.st->done) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = blockIdx.x * kDampWarps + wid; i < P.nc; i += gridDim.x * kDampWarps) {
        double *A = sA[wid];
        __syncwarp();
        for (int e = lane; e < 81; e += 32) {
            const int a = e / 9, b = e - 9 * (e / 9);
            double sum = 0.0;
            for (int c = cfirst[i]; c < cfirst[i + 1]; ++c) sum += P.cpart[54 * (int64_t)c + sym9(a, b)];
            A[e] = P.Bd[81 * (int64_t)i + e] - sum;
        }
        __syncwarp();
        warp_spd_inverse9(A, sY[wid], sil[wid], P.Binv + 81 * (int64_t)i);  // not PD: B~_i^-1 stays
    }
}

// ---------------------------------------------------------------------------
// shared pieces of the point-major passes
// ---------------------------------------------------------------------------

// Streaming variant: evict-first loads, so the once-per-pass Jacobian stream
// does not push the per-observation s vectors and camera data out of L2.
template <typename T>
__device__ __forceinline__ void load_jac_stream(const T *__restrict__ J, int64_t npad, int64_t o, T *Jc, T *Jp) {
#pragma unroll
    for (int q = 0; q < 18; ++q) Jc[q] = __ldcs(J + q * npad + o);
#pragma unroll
    for (int q = 0; q < 6; ++q) Jp[q] = __ldcs(J + (18 + q) * npad + o);
}

template <typename T>
__device__ __forceinline__ void sym3_apply(const T *__restrict__ C, T a0, T a1, T a2, T *b) {
    const T c0 = __ldg(C), c1 = __ldg(C + 1), c2 = __ldg(C + 2), c3 = __ldg(C + 3), c4 = __ldg(C + 4),
            c5 = __ldg(C + 5);
    b[0] = c0 * a0 + c1 * a1 + c2 * a2;
    b[1] = c1 * a0 + c3 * a1 + c4 * a2;
    b[2] = c2 * a0 + c4 * a1 + c5 * a2;
}

// ---------------------------------------------------------------------------
// The implicit Schur product S p = B~ p - E C~^-1 E^T p in two passes per PCG
// iteration, neither of which writes to a shared accumulator:
//  * point pass (point-major, warp chunks of whole points, <= 32
//    observations): b_j = C~_j^-1 sum_k Jp~_k^T Jc~_k p_i(k) by a segmented
//    shuffle scan, then s_k = Jp~_k b_j is stored per observation;
//  * camera pass (camera-major, one warp per camera chunk of <= 1024
//    observations): the chunk's sum of Jc~_k^T s_k; the last warp to finish a
//    camera adds that camera's chunk sums in a fixed order and forms
//    q_i = B~_i p_i - c_i (or the right-hand side g_i = v_i - c_i).
// In FP32-mixed the camera pass recomputes Jc~ from the camera table and the
// point (camera-uniform per warp, cheaper than streaming 72 bytes again); the
// FP64 form streams a camera-major copy written at linearisation.
// ---------------------------------------------------------------------------
template <typename T>
struct V2;
template <>
struct V2<float> {
    using type = float2;
};
template <>
struct V2<double> {
    using type = double2;
};

template <typename T>
__device__ __forceinline__ void gather_p(const T *ps, const T *pT, int cam, T *pa) {
    if (ps) {
#pragma unroll
        for (int a = 0; a < 9; ++a) pa[a] = ps[cam * 9 + a];
    } else {
        const T *pv = pT + (int64_t)cam * kVec;
#pragma unroll
        for (int a = 0; a < 9; ++a) pa[a] = ldcg(pv + a);
    }
}

// E^T p contribution of one observation: u = Jp^T (Jc p)
template <typename T>
__device__ __forceinline__ void et_p(const T *Jc, const T *Jp, const T *pa, T *u) {
    T t0 = T(0), t1 = T(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        t0 += Jc[a] * pa[a];
        t1 += Jc[9 + a] * pa[a];
    }
    u[0] = Jp[0] * t0 + Jp[3] * t1;
    u[1] = Jp[1] * t0 + Jp[4] * t1;
    u[2] = Jp[2] * t0 + Jp[5] * t1;
}

template <typename T>
__device__ __forceinline__ void load_sym3(const T *__restrict__ C, T *c) {
#pragma unroll
    for (int q = 0; q < 6; ++q) c[q] = __ldg(C + q);
}
template <typename T>
__device__ __forceinline__ void apply_sym3(const T *c, T a0, T a1, T a2, T *b) {
    b[0] = c[0] * a0 + c[1] * a1 + c[2] * a2;
    b[1] = c[1] * a0 + c[3] * a1 + c[4] * a2;
    b[2] = c[2] * a0 + c[4] * a1 + c[5] * a2;
}

template <typename T>
__device__ __forceinline__ void store_s(typename V2<T>::type *sbuf, int64_t o, const T *Jp, const T *b) {
    typename V2<T>::type v;
    v.x = Jp[0] * b[0] + Jp[1] * b[1] + Jp[2] * b[2];
    v.y = Jp[3] * b[0] + Jp[4] * b[1] + Jp[5] * b[2];
    sbuf[o] = v;
}

// Point pass.  RHS: b_j = C~_j^-1 w_j.  Otherwise b_j = C~_j^-1 sum_k u_k.
template <typename T, bool RHS>
__device__ void point_pass(const Prob &P, const T *ps, const T *pT, typename V2<T>::type *sbuf) {
    const T *__restrict__ J = (const T *)P.J;
    const T *__restrict__ Cinv = (const T *)P.Cinv;
    const int64_t npad = P.npad;
    const int lane = threadIdx.x & 31;
    const int nwarp = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;
    const int gstride = gridDim.x * nwarp;
    int w = blockIdx.x * nwarp + (threadIdx.x >> 5);
    int2 c0 = make_int2(0, 0), c1 = make_int2(0, 0);
    if (w < P.n_wchunks) {
        c0 = P.wchunk[w];
        c1 = P.wchunk[w + 1];
    }
    for (; w < P.n_wchunks; w += gstride) {
        const int wn = w + gstride;
        int2 n0 = c0, n1 = c1;
        if (wn < P.n_wchunks) {
            n0 = P.wchunk[wn];
            n1 = P.wchunk[wn + 1];
        }
        const int o0 = c0.y, m = c1.y - c0.y;
        if (m <= 32) {
            const bool act = lane < m;
            const int64_t o = (int64_t)o0 + (act ? lane : 0);
            // point of each lane from the chunk's point starts (whole points, <= 32 observations)
            const int npts = c1.x - c0.x;
            const int rs = lane < npts ? __ldg(P.pt_ptr + c0.x + lane) - o0 : 32;
            const unsigned starts = __reduce_or_sync(full, rs < 32 ? (1u << rs) : 0u);
            const int pt = act ? c0.x + __popc(starts & (0xffffffffu >> (31 - lane))) - 1 : -1 - lane;
            const int cam = act ? __ldcs(P.pm_cam + o) : 0;
            const int so = act ? __ldcs(P.pm2cm + o) : 0;  // where the camera pass reads s
            T Jc[18], Jp[6], ci[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) Jp[q] = ci[q] = T(0);
#pragma unroll
            for (int q = 0; q < 18; ++q) Jc[q] = T(0);
            if (act) {
#pragma unroll
                for (int q = 0; q < 6; ++q) Jp[q] = __ldcs(J + (18 + q) * npad + o);
                if (!RHS)
#pragma unroll
                    for (int q = 0; q < 18; ++q) Jc[q] = __ldcs(J + q * npad + o);
                load_sym3(Cinv + 6 * (int64_t)pt, ci);
            }
            T b[3] = {T(0), T(0), T(0)};
            if (RHS) {
                if (act)
                    apply_sym3(ci, (T)P.w[3 * (int64_t)pt], (T)P.w[3 * (int64_t)pt + 1], (T)P.w[3 * (int64_t)pt + 2],
                               b);
            } else {
                T u[3] = {T(0), T(0), T(0)};
                if (act) {
                    T pa[9];
                    gather_p(ps, pT, cam, pa);
                    et_p(Jc, Jp, pa, u);
                }
                // inclusive segmented scan keyed by point (segments are contiguous).
                // FP64: only as many levels as the chunk's longest point needs
                // (each level is three warp-wide FP64 adds on the FP64 pipe)
                int span = 32;
                if constexpr (sizeof(T) == 8) {
                    const int nrs = __shfl_down_sync(full, rs, 1);
                    const int len = lane < npts ? (lane + 1 < npts ? nrs : m) - rs : 0;
                    span = __reduce_max_sync(full, len);
                }
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    if (d >= span) break;
                    const int kp = __shfl_up_sync(full, pt, d);
                    const T v0 = __shfl_up_sync(full, u[0], d), v1 = __shfl_up_sync(full, u[1], d),
                            v2 = __shfl_up_sync(full, u[2], d);
                    if (lane >= d && kp == pt) {
                        u[0] += v0;
                        u[1] += v1;
                        u[2] += v2;
                    }
                }
                const int nxt = __shfl_down_sync(full, pt, 1);
                const bool tail = act && (lane == 31 || lane == m - 1 || nxt != pt);
                const unsigned tails = __ballot_sync(full, tail);
                T bt[3];
                apply_sym3(ci, u[0], u[1], u[2], bt);
                const unsigned mine = tails & (0xffffffffu << lane);
                const int src = mine ? __ffs(mine) - 1 : lane;
                b[0] = __shfl_sync(full, bt[0], src);
                b[1] = __shfl_sync(full, bt[1], src);
                b[2] = __shfl_sync(full, bt[2], src);
            }
            if (act) store_s<T>(sbuf, so, Jp, b);
        } else {
            // one point with a long track: two sweeps over 32-observation slices
            const int pt = c0.x;
            T ci[6], b[3];
            load_sym3(Cinv + 6 * (int64_t)pt, ci);
            if (RHS) {
                apply_sym3(ci, (T)P.w[3 * (int64_t)pt], (T)P.w[3 * (int64_t)pt + 1], (T)P.w[3 * (int64_t)pt + 2], b);
            } else {
                T a[3] = {T(0), T(0), T(0)};
                for (int base = 0; base < m; base += 32) {
                    if (base + lane < m) {
                        const int64_t o = (int64_t)o0 + base + lane;
                        T Jc[18], Jp[6], pa[9], u[3];
                        load_jac_stream(J, npad, o, Jc, Jp);
                        gather_p(ps, pT, __ldcs(P.pm_cam + o), pa);
                        et_p(Jc, Jp, pa, u);
                        a[0] += u[0];
                        a[1] += u[1];
                        a[2] += u[2];
                    }
                }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) {
                    a[0] += __shfl_xor_sync(full, a[0], d);
                    a[1] += __shfl_xor_sync(full, a[1], d);
                    a[2] += __shfl_xor_sync(full, a[2], d);
                }
                apply_sym3(ci, a[0], a[1], a[2], b);
            }
            for (int base = 0; base < m; base += 32) {
                if (base + lane < m) {
                    const int64_t o = (int64_t)o0 + base + lane;
                    T Jp[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q) Jp[q] = __ldcs(J + (18 + q) * npad + o);
                    store_s<T>(sbuf, __ldcs(P.pm2cm + o), Jp, b);
                }
            }
        }
        c0 = n0;
        c1 = n1;
    }
}


// ---------------------------------------------------------------------------
// Factored FP32 form (analytic Jacobian).  With P = R X + t the camera-frame
// point, p = -(P_x, P_y) / P_z, r2 = |p|^2, d = 1 + k1 r2 + k2 r2^2 and
// A = f (d I + (2 k1 + 4 k2 r2) p p^T), the BAL Jacobian of one observation is
//   D = d(pixel)/dP = -(1/P_z) A [I | p],   Jp = D R,   Jc = [-D R [X]x M | D | p (d, f r2, f r2^2)]
// (M: the rotation factor of the camera table).  Because R (a x b) = R a x R b,
// the two products the PCG needs reduce to per-observation data and
// per-camera constants:
//   Jc v = D (n x (P - t) + v_t) + p (d v_f + f r2 v_k1 + f r2^2 v_k2),   n = R M v_w,
//   sum_k Jc_k^T s_k = [ (R M)^T sum_k RX_k x D_k^T s_k ; sum_k D_k^T s_k ;
//                        (sum_k d p.s, f sum_k r2 p.s, f sum_k r2^2 p.s) ],
// RX = R X = P - t.  The point pass streams (px, py, 1/P_z) and W Jp, 36 bytes
// per observation instead of the 96-byte Jacobian, and forms
// (n x (P - t) + v_t) / P_z = n x (-px, -py, 1) + h / P_z with the camera
// constant h = v_t - n x t: one cancellation of order |t| / |RX| per
// observation.  The camera pass reads (RX, 1/P_z) as one float4 and recomputes
// p from P = RX + t, so its cross products, summed over a chunk of hundreds of
// observations, use RX itself: forming them as P_z q - t instead would cancel
// after the sum, and that loss broke the PCG near mu ~ 1e-7.
// (In the first-order rotation branch, |w|^2 <= 2.2e-16, both apply
// R = I + [w]x where the Jacobian has I: a relative difference of at most |w|,
// below FP32 rounding.)
//
// Per-camera row of kRow = 12 floats for a vector v = (v_w, v_t, v_f, v_k1, v_k2):
//   n = R M v_w, h = v_t - n x t, e = (v_f, f v_k1, f v_k2), then (f, k1, k2)
//   (consts) or zeros.  The row is linear in v apart from the constants, so
//   row(z) + beta row(p) with the constants carried by row(z) alone is the row
//   of z + beta p.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fact_row(const float *__restrict__ ct, const float *v, bool consts, float *r) {
    const float m0 = ct[9] * v[0] + ct[10] * v[1] + ct[11] * v[2];
    const float m1 = ct[12] * v[0] + ct[13] * v[1] + ct[14] * v[2];
    const float m2 = ct[15] * v[0] + ct[16] * v[1] + ct[17] * v[2];
    const float n0 = ct[0] * m0 + ct[1] * m1 + ct[2] * m2;
    const float n1 = ct[3] * m0 + ct[4] * m1 + ct[5] * m2;
    const float n2 = ct[6] * m0 + ct[7] * m1 + ct[8] * m2;
    const float t0 = ct[18], t1 = ct[19], t2 = ct[20], f = ct[21];
    r[0] = n0;
    r[1] = n1;
    r[2] = n2;
    r[3] = v[3] - (n1 * t2 - n2 * t1);
    r[4] = v[4] - (n2 * t0 - n0 * t2);
    r[5] = v[5] - (n0 * t1 - n1 * t0);
    r[6] = v[6];
    r[7] = f * v[7];
    r[8] = f * v[8];
    r[9] = consts ? f : 0.f;
    r[10] = consts ? ct[22] : 0.f;
    r[11] = consts ? ct[23] : 0.f;
}

// Warp-collective (all 32 lanes call it): lanes 9s..9s+8 hold the nine
// components of camera `cam` (lane s of the three-camera group); each active
// lane writes its element of the camera's row to dst[cam][kRow] (lanes of rows
// 0..2 also the elements 9..11).
__device__ __forceinline__ void fact_row_store(const Prob &P, float *dst, int cam, bool act, double val, int sub,
                                               int row, bool consts) {
    const float fv = (float)val;
    float v[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) v[j] = __shfl_sync(0xffffffffu, fv, (9 * sub + j) & 31);
    if (!act) return;
    float r[kRow];
    fact_row((const float *)P.camtab + (int64_t)cam * kCamTab, v, consts, r);
    float mine = r[0], pad = r[9];
#pragma unroll
    for (int j = 1; j < 9; ++j)
        if (row == j) mine = r[j];
    if (row == 1) pad = r[10];
    if (row == 2) pad = r[11];
    stcg(dst + (int64_t)cam * kRow + row, mine);
    if (row < 3) stcg(dst + (int64_t)cam * kRow + 9 + row, pad);
}

// The camera's row: shared memory (ps, [nc][kRow]) or the global copy.
__device__ __forceinline__ void gather_row(const float *ps, const float *pT, int cam, float *r) {
    float4 q[kRow / 4];
    if (ps) {
        const float4 *src = (const float4 *)(ps + cam * kRow);
#pragma unroll
        for (int i = 0; i < kRow / 4; ++i) q[i] = src[i];
    } else {
        const float4 *src = (const float4 *)(pT + (int64_t)cam * kRow);
#pragma unroll
        for (int i = 0; i < kRow / 4; ++i) q[i] = __ldcg(src + i);
    }
#pragma unroll
    for (int i = 0; i < kRow / 4; ++i) {
        r[4 * i] = q[i].x;
        r[4 * i + 1] = q[i].y;
        r[4 * i + 2] = q[i].z;
        r[4 * i + 3] = q[i].w;
    }
}

// t = Jc v (unscaled) for one observation from (px, py, 1/Pz) and the camera's row.
__device__ __forceinline__ void fact_jc_v(float px, float py, float iz, const float *r, float *t) {
    const float f = r[9], k1 = r[10], k2 = r[11];
    const float r2 = px * px + py * py;
    const float d = 1.f + k1 * r2 + k2 * r2 * r2;
    const float dd = 2.f * k1 + 4.f * k2 * r2;
    const float a00 = f * (d + dd * px * px), a01 = f * dd * px * py, a11 = f * (d + dd * py * py);
    // (n x (P - t) + v_t) / P_z = n x (-px, -py, 1) + h / P_z
    const float w0 = r[1] + r[2] * py + iz * r[3];
    const float w1 = -r[0] - r[2] * px + iz * r[4];
    const float w2 = r[1] * px - r[0] * py + iz * r[5];
    const float z0 = w0 + px * w2, z1 = w1 + py * w2;
    const float ei = r[6] * d + r2 * (r[7] + r2 * r[8]);
    t[0] = -(a00 * z0 + a01 * z1) + px * ei;
    t[1] = -(a01 * z0 + a11 * z1) + py * ei;
}

// One point with a long track (more than 32 observations, one warp): two
// sweeps over 32-observation slices, reading global memory.
template <bool RHS>
__device__ void long_chunk_fact(const Prob &P, const float *ps, const float *pT, float2 *sbuf, int pt, int o0, int m) {
    const float *__restrict__ Jh = P.Jph;
    const float *__restrict__ PX = P.PXpm;
    const int64_t npad = P.npad;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    float ci[6], b[3];
    load_sym3((const float *)P.Cinv + 6 * (int64_t)pt, ci);
    if (RHS) {
        apply_sym3(ci, (float)P.w[3 * (int64_t)pt], (float)P.w[3 * (int64_t)pt + 1], (float)P.w[3 * (int64_t)pt + 2],
                   b);
    } else {
        float a[3] = {0.f, 0.f, 0.f};
        for (int base = 0; base < m; base += 32) {
            if (base + lane < m) {
                const int64_t o = (int64_t)o0 + base + lane;
                float r[kRow], t[2];
                gather_row(ps, pT, __ldcs(P.pm_cam + o), r);
                fact_jc_v(__ldcs(PX + o), __ldcs(PX + npad + o), __ldcs(PX + 2 * npad + o), r, t);
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    a[q] += __ldcs(Jh + q * npad + o) * t[0] + __ldcs(Jh + (3 + q) * npad + o) * t[1];
            }
        }
#pragma unroll
        for (int dl = 16; dl > 0; dl >>= 1) {
            a[0] += __shfl_xor_sync(full, a[0], dl);
            a[1] += __shfl_xor_sync(full, a[1], dl);
            a[2] += __shfl_xor_sync(full, a[2], dl);
        }
        apply_sym3(ci, a[0], a[1], a[2], b);
    }
    for (int base = 0; base < m; base += 32) {
        if (base + lane < m) {
            const int64_t o = (int64_t)o0 + base + lane;
            float jh[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) jh[q] = __ldcs(Jh + q * npad + o);
            store_s<float>(sbuf, __ldcs(P.pm2cm + o), jh, b);
        }
    }
}

// Point pass of the factored form: as point_pass, with u = (W Jp)^T (Jc p)
// and s = (W Jp) b, so the camera pass forms sum Jc^T s with unscaled Jc.
template <bool RHS>
__device__ void point_pass_fact(const Prob &P, const float *ps, const float *pT, float2 *sbuf) {
    const float *__restrict__ Jh = P.Jph;
    const float *__restrict__ PX = P.PXpm;
    const float *__restrict__ Cinv = (const float *)P.Cinv;
    const int64_t npad = P.npad;
    const int lane = threadIdx.x & 31;
    const int nwarp = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;
    const int gstride = gridDim.x * nwarp;
    int w = blockIdx.x * nwarp + (threadIdx.x >> 5);
    int2 c0 = make_int2(0, 0), c1 = make_int2(0, 0);
    if (w < P.n_wchunks) {
        c0 = P.wchunk[w];
        c1 = P.wchunk[w + 1];
    }
    for (; w < P.n_wchunks; w += gstride) {
        const int wn = w + gstride;
        int2 n0 = c0, n1 = c1;
        if (wn < P.n_wchunks) {
            n0 = P.wchunk[wn];
            n1 = P.wchunk[wn + 1];
        }
        const int o0 = c0.y, m = c1.y - c0.y;
        if (m <= 32) {
            const bool act = lane < m;
            const int64_t o = (int64_t)o0 + (act ? lane : 0);
            // point of each lane from the chunk's point starts (whole points, <= 32 observations)
            const int npts = c1.x - c0.x;
            const int rs = lane < npts ? __ldg(P.pt_ptr + c0.x + lane) - o0 : 32;
            const unsigned starts = __reduce_or_sync(full, rs < 32 ? (1u << rs) : 0u);
            const int pt = act ? c0.x + __popc(starts & (0xffffffffu >> (31 - lane))) - 1 : -1 - lane;
            const int cam = act ? __ldcs(P.pm_cam + o) : 0;
            const int so = act ? __ldcs(P.pm2cm + o) : 0;  // where the camera pass reads s
            float jh[6], ci[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) jh[q] = ci[q] = 0.f;
            float px = 0.f, py = 0.f, iz = 0.f;
            if (act) {
#pragma unroll
                for (int q = 0; q < 6; ++q) jh[q] = __ldcs(Jh + q * npad + o);
                if (!RHS) {
                    px = __ldcs(PX + o);
                    py = __ldcs(PX + npad + o);
                    iz = __ldcs(PX + 2 * npad + o);
                }
                load_sym3(Cinv + 6 * (int64_t)pt, ci);
            }
            float b[3] = {0.f, 0.f, 0.f};
            if (RHS) {
                if (act)
                    apply_sym3(ci, (float)P.w[3 * (int64_t)pt], (float)P.w[3 * (int64_t)pt + 1],
                               (float)P.w[3 * (int64_t)pt + 2], b);
            } else {
                float u[3] = {0.f, 0.f, 0.f};
                if (act) {
                    float r[kRow], t[2];
                    gather_row(ps, pT, cam, r);
                    fact_jc_v(px, py, iz, r, t);
                    u[0] = jh[0] * t[0] + jh[3] * t[1];
                    u[1] = jh[1] * t[0] + jh[4] * t[1];
                    u[2] = jh[2] * t[0] + jh[5] * t[1];
                }
                // inclusive segmented scan keyed by point (segments are contiguous)
#pragma unroll
                for (int dl = 1; dl < 32; dl <<= 1) {
                    const int kp = __shfl_up_sync(full, pt, dl);
                    const float v0 = __shfl_up_sync(full, u[0], dl), v1 = __shfl_up_sync(full, u[1], dl),
                                v2 = __shfl_up_sync(full, u[2], dl);
                    if (lane >= dl && kp == pt) {
                        u[0] += v0;
                        u[1] += v1;
                        u[2] += v2;
                    }
                }
                const int nxt = __shfl_down_sync(full, pt, 1);
                const bool tail = act && (lane == 31 || lane == m - 1 || nxt != pt);
                const unsigned tails = __ballot_sync(full, tail);
                float bt[3];
                apply_sym3(ci, u[0], u[1], u[2], bt);
                const unsigned mine = tails & (0xffffffffu << lane);
                const int src = mine ? __ffs(mine) - 1 : lane;
                b[0] = __shfl_sync(full, bt[0], src);
                b[1] = __shfl_sync(full, bt[1], src);
                b[2] = __shfl_sync(full, bt[2], src);
            }
            if (act) store_s<float>(sbuf, so, jh, b);
        } else {
            long_chunk_fact<RHS>(P, ps, pT, sbuf, c0.x, o0, m);
        }
        c0 = n0;
        c1 = n1;
    }
}

// ---------------------------------------------------------------------------
// Staged point pass of the factored form (iterations and the single product;
// the right-hand-side pass keeps point_pass_fact).  A producer/consumer
// pipeline in shared memory: the CTA's last warp copies the CTA's tiles (tile t
// belongs to CTA t mod grid) into S stages with 1-D bulk copies, each stage
// completing on its "full" mbarrier; the other warps wait for a stage, work on
// it from shared memory (one warp chunk each), and release it on its "empty"
// mbarrier, which the producer waits on before refilling the stage.  There is no
// CTA-wide barrier between tiles, so warps drift across tiles and the copies run
// up to S tiles ahead of the slowest consumer.  The per-observation streams do
// not change within a launch, so the producer also runs ahead into the next
// pass, across the camera pass and the grid barriers.  Use index u of the CTA
// (counted over the whole launch) lives in stage u mod S; its full phase has
// parity (u / S) mod 2, and so has the empty phase that releases it.
// ---------------------------------------------------------------------------
struct StageOrg {
    int32_t oa, ca, pa, wa;  // first index copied of the observation rows, C~^-1 floats, pt_ptr, chunk table
    int32_t cb, ce;          // the tile's chunks [cb, ce)
    int32_t ok, pad;         // 0: the tile did not fit its stage (not copied)
};
constexpr long long kStageSpin = 1ll << 20;  // polls of a stage barrier before giving up

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Producer warp (all lanes): the copies of use `use` into stage use mod S, one
// array per lane; d0..d2 is the tile's descriptor (in every lane).
__device__ void stage_issue(const Prob &P, unsigned char *stages, uint64_t *full, StageOrg *org, int S, uint32_t use,
                            int4 d0, int4 d1, int4 d2) {
    const int lane = threadIdx.x & 31;
    const int sidx = (int)(use % (uint32_t)S);
    const int oa = d0.x, ob = d0.y, ca = d0.z, cz = d0.w, pa = d1.x, pz = d1.y, wa = d1.z, wz = d1.w;
    const bool fits = d2.y > d2.x && ob - oa <= kTileRow && cz - ca <= 6 * kTilePts + 8 && pz - pa <= kTilePts + 8 &&
                      wz - wa <= kTileChunks + 4 && d2.y - d2.x <= kTileChunks;
    const uint32_t bo = 4u * (uint32_t)(ob - oa);
    uint64_t *bar = full + sidx;
    float *st = (float *)(stages + (size_t)sidx * kStageBytes);
    if (lane == 0) {
        org[sidx] = StageOrg{oa, ca, pa, wa, d2.x, d2.y, fits ? 1 : 0, 0};
        const uint32_t total = 11u * bo + 4u * (uint32_t)(cz - ca) + 4u * (uint32_t)(pz - pa) + 8u * (uint32_t)(wz - wa);
        mbar_arrive_expect_tx(bar, fits ? total : 0u);
    }
    __syncwarp();
    if (!fits || lane >= 14) return;
    const void *src;
    void *dst;
    uint32_t bytes = bo;
    if (lane == 0) {
        src = P.pm_cam + oa;
        dst = st;
    } else if (lane == 1) {
        src = P.pm2cm + oa;
        dst = st + kStwSo;
    } else if (lane < 8) {
        src = P.Jph + (int64_t)(lane - 2) * P.npad + oa;
        dst = st + kStwJh + (lane - 2) * kTileRow;
    } else if (lane < 11) {
        src = P.PXpm + (int64_t)(lane - 8) * P.npad + oa;
        dst = st + kStwPx + (lane - 8) * kTileRow;
    } else if (lane == 11) {
        src = (const float *)P.Cinv + ca;
        dst = st + kStwCinv;
        bytes = 4u * (uint32_t)(cz - ca);
    } else if (lane == 12) {
        src = P.pt_ptr + pa;
        dst = st + kStwPtp;
        bytes = 4u * (uint32_t)(pz - pa);
    } else {
        src = P.wchunk + wa;
        dst = st + kStwWch;
        bytes = 8u * (uint32_t)(wz - wa);
    }
    bulk_g2s(dst, src, bytes, bar);
}

// The arithmetic of one warp chunk (at most 32 observations) once its inputs
// are in registers: t = Jc p from the camera row, u = (W Jp)^T t, the
// segmented scan by point, b = C~^-1 u at each point's last lane, and
// s = (W Jp) b written to the camera-major position so.
__device__ __forceinline__ void chunk_tail(const float *ps, const float *pT, float2 *sbuf, bool act, int m, int pt,
                                           int cam, int so, const float *jh, const float *ci, float px, float py,
                                           float iz) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    float u[3] = {0.f, 0.f, 0.f};
    if (act) {
        float r[kRow], t[2];
        gather_row(ps, pT, cam, r);
        fact_jc_v(px, py, iz, r, t);
        u[0] = jh[0] * t[0] + jh[3] * t[1];
        u[1] = jh[1] * t[0] + jh[4] * t[1];
        u[2] = jh[2] * t[0] + jh[5] * t[1];
    }
    // inclusive segmented scan keyed by point (segments are contiguous)
#pragma unroll
    for (int dl = 1; dl < 32; dl <<= 1) {
        const int kp = __shfl_up_sync(full, pt, dl);
        const float v0 = __shfl_up_sync(full, u[0], dl), v1 = __shfl_up_sync(full, u[1], dl),
                    v2 = __shfl_up_sync(full, u[2], dl);
        if (lane >= dl && kp == pt) {
            u[0] += v0;
            u[1] += v1;
            u[2] += v2;
        }
    }
    const int nxt = __shfl_down_sync(full, pt, 1);
    const bool tail = act && (lane == 31 || lane == m - 1 || nxt != pt);
    const unsigned tails = __ballot_sync(full, tail);
    float bt[3], b[3];
    apply_sym3(ci, u[0], u[1], u[2], bt);
    const unsigned mine = tails & (0xffffffffu << lane);
    const int src = mine ? __ffs(mine) - 1 : lane;
    b[0] = __shfl_sync(full, bt[0], src);
    b[1] = __shfl_sync(full, bt[1], src);
    b[2] = __shfl_sync(full, bt[2], src);
    if (act) store_s<float>(sbuf, so, jh, b);
}

// One warp chunk of a stage (at most 32 observations), as point_pass_fact with
// every per-observation and per-point input read from the stage.
__device__ __forceinline__ void staged_chunk(const float *ps, const float *pT, float2 *sbuf, const float *st,
                                             const StageOrg &o, int k) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int *s_cam = (const int *)st, *s_so = (const int *)(st + kStwSo);
    const float *s_jh = st + kStwJh, *s_px = st + kStwPx, *s_ci = st + kStwCinv;
    const int *s_ptp = (const int *)(st + kStwPtp);
    const int2 *s_wch = (const int2 *)(st + kStwWch);
    const int2 c0 = s_wch[k - o.wa], c1 = s_wch[k + 1 - o.wa];
    const int o0 = c0.y, m = c1.y - c0.y;  // at most 32: longer tracks are not in tiles
    const bool act = lane < m;
    const int li = o0 - o.oa + (act ? lane : 0);
    const int npts = c1.x - c0.x;
    const int rs = lane < npts ? s_ptp[c0.x + lane - o.pa] - o0 : 32;
    const unsigned starts = __reduce_or_sync(full, rs < 32 ? (1u << rs) : 0u);
    const int pt = act ? c0.x + __popc(starts & (0xffffffffu >> (31 - lane))) - 1 : -1 - lane;
    float jh[6], ci[6], px = 0.f, py = 0.f, iz = 0.f;
    int so = 0, cam = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) jh[q] = ci[q] = 0.f;
    if (act) {
        so = s_so[li];
        cam = s_cam[li];
#pragma unroll
        for (int q = 0; q < 6; ++q) jh[q] = s_jh[q * kTileRow + li];
        // C~^-1 of the point, from the stage (plain shared-memory loads)
#pragma unroll
        for (int q = 0; q < 6; ++q) ci[q] = s_ci[6 * pt - o.ca + q];
        px = s_px[li];
        py = s_px[kTileRow + li];
        iz = s_px[2 * kTileRow + li];
    }
    chunk_tail(ps, pT, sbuf, act, m, pt, cam, so, jh, ci, px, py, iz);
}

// The staged pass.  `base` counts the uses consumed before this pass (the same
// in every thread); `issued` the uses issued so far (the producer warp's).
// Returns false in every thread if a stage barrier gave up (the error is recorded).
__device__ bool point_pass_fact_staged(const Prob &P, const float *ps, const float *pT, float2 *sbuf,
                                       unsigned char *stages, uint64_t *full, uint64_t *empty, StageOrg *org, int S,
                                       int my_nt, uint32_t &base, uint32_t &issued) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const uint32_t Su = (uint32_t)S;
    bool ok = true;
    if (wid == nwarp - 1) {
        // producer: through the first S uses of the next pass, each after the
        // consumers released its stage (the tile's descriptor is read first, so
        // its latency overlaps the wait)
        const uint32_t target = my_nt > 0 ? base + (uint32_t)my_nt + Su : 0u;
        while (issued < target) {
            const uint32_t u = issued;
            const int t = (int)blockIdx.x + (int)(u % (uint32_t)my_nt) * (int)gridDim.x;
            int4 d = make_int4(0, 0, 0, 0);
            if (lane < 3) d = __ldg(P.tdesc + 3 * (int64_t)t + lane);
            if (u >= Su && !mbar_wait(empty + u % Su, (u / Su - 1u) & 1u, kStageSpin)) {
                if (lane == 0) atomicCAS(&P.st->err, 0, (int)MBA_ERR_TIMEOUT);
                ok = false;
                break;
            }
            int4 d0, d1, d2;
            d0.x = __shfl_sync(0xffffffffu, d.x, 0), d0.y = __shfl_sync(0xffffffffu, d.y, 0);
            d0.z = __shfl_sync(0xffffffffu, d.z, 0), d0.w = __shfl_sync(0xffffffffu, d.w, 0);
            d1.x = __shfl_sync(0xffffffffu, d.x, 1), d1.y = __shfl_sync(0xffffffffu, d.y, 1);
            d1.z = __shfl_sync(0xffffffffu, d.z, 1), d1.w = __shfl_sync(0xffffffffu, d.w, 1);
            d2.x = __shfl_sync(0xffffffffu, d.x, 2), d2.y = __shfl_sync(0xffffffffu, d.y, 2);
            d2.z = 0, d2.w = 0;
            stage_issue(P, stages, full, org, S, u, d0, d1, d2);
            ++issued;
        }
    } else {
        // consumers: warp w works chunk w of every tile, then releases the stage
        for (int j = 0; j < my_nt; ++j) {
            const uint32_t u = base + (uint32_t)j;
            const int sidx = (int)(u % Su);
            if (!mbar_wait(full + sidx, (u / Su) & 1u, kStageSpin)) {
                if (lane == 0) atomicCAS(&P.st->err, 0, (int)MBA_ERR_TIMEOUT);
                ok = false;
                break;
            }
            const StageOrg o = org[sidx];
            if (o.ok) {
                const int k = o.cb + wid;
                if (k < o.ce) staged_chunk(ps, pT, sbuf, (const float *)(stages + (size_t)sidx * kStageBytes), o, k);
            } else if (wid == 0 && lane == 0) {
                atomicCAS(&P.st->err, 0, (int)MBA_ERR_INVALID_ARG);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + sidx);
        }
    }
    base += (uint32_t)my_nt;
    // chunks of tracks longer than 32 observations, over every warp of the grid
    if (ok)
        for (int i = (int)blockIdx.x * nwarp + wid; i < P.n_long; i += (int)gridDim.x * nwarp) {
            const int k = P.long_chunks[i];
            const int2 c0 = P.wchunk[k], c1 = P.wchunk[k + 1];
            long_chunk_fact<false>(P, ps, pT, sbuf, c0.x, c0.y, c1.y - c0.y);
        }
    return __syncthreads_or(ok ? 0 : 1) == 0;
}

template <typename T, bool RHS, bool FACT>
__device__ __forceinline__ void point_pass_any(const Prob &P, const T *ps, const T *pT, typename V2<T>::type *sbuf) {
    if constexpr (FACT) point_pass_fact<RHS>(P, (const float *)ps, (const float *)pT, (float2 *)sbuf);
    else point_pass<T, RHS>(P, ps, pT, sbuf);
}

// Stored form (FP64, and FP32-mixed with dual-number Jacobians): acc += Jc~^T s
// as 18 fused multiply-adds on the stored camera-major Jc~ (sqrt(W) included).
template <typename T>
__device__ __forceinline__ void camera_acc_stored(const Prob &P, int64_t s, T s0, T s1, T *acc) {
    const T *__restrict__ Jc = (const T *)P.JcmT;
#pragma unroll
    for (int a = 0; a < 9; ++a)
        acc[a] = fma(__ldcs(Jc + a * P.npad + s), s0, fma(__ldcs(Jc + (9 + a) * P.npad + s), s1, acc[a]));
}

enum CamMode { CAM_RHS = 0, CAM_ITER = 1, CAM_MATVEC = 2, CAM_SR = 3 };

__device__ __forceinline__ double2 cta_sum2(double x, double y, bool warp_data, double *sb);
__device__ __forceinline__ double3 cta_sum3(double x, double y, double z, bool warp_data, double *sb);


// Camera pass.  Each CTA owns a contiguous run of whole cameras
// [cta_cam[b], cta_cam[b+1]), balanced by observation count at creation; its
// warps reduce the run's camera chunks into shared-memory slots, then, after a
// block barrier, each camera's chunk sums are added in chunk order and the
// camera is finalised.  No global atomics or fences; results do not depend on
// timing.  CAM_RHS: g = v - c, x = 0, r = g, z = B~^-1 g; returns this CTA's
// (r.r, r.z).  CAM_ITER: p = z + beta p_prev (p = z first), q = B~ p - c;
// returns (p.q, 0).  CAM_MATVEC: q = B~ p - c with p given.  CAM_SR (the
// single-reduction PCG): w = B~ u - c with u in P.z, into P.q; returns (r.r,
// r.u) and w.u in *third.
template <typename T, int MODE, bool JS>
__device__ double2 camera_pass(const Prob &P, const typename V2<T>::type *sbuf, const double *p_prev, double *p_cur,
                               T *pT_cur, double beta, bool first, double *cslot, double *sb,
                               double *third = nullptr) {
    using T2 = typename V2<T>::type;
    constexpr int U = 4;
    constexpr bool FACT = sizeof(T) == 4 && !JS;
    __shared__ T cts[32][kCamTab];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwarp = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;
    const T *camtab = (const T *)P.camtab;
    T *ct = cts[wid];
    __shared__ int next_chunk;
    const int cb = P.cta_cam[blockIdx.x], ce = P.cta_cam[blockIdx.x + 1];
    const int k0 = P.cfirst[cb], k1 = P.cfirst[ce];
    if (threadIdx.x == 0) next_chunk = k0 + nwarp;
    __syncthreads();
    int loaded = -1;
    // warps claim chunks dynamically; each chunk's sum goes to its own slot, so
    // the result does not depend on which warp took it
    for (int k = k0 + wid; k < k1;) {
        const int cam = P.cchunk_cam[k];
        const int b0 = P.cchunk_beg[k], b1 = P.cchunk_beg[k + 1];
        if (sizeof(T) == 4 && !JS && cam != loaded) {
            __syncwarp();
            if (lane < kCamTab) ct[lane] = __ldg(camtab + (int64_t)cam * kCamTab + lane);
            __syncwarp();
            loaded = cam;
        }
        T acc[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = T(0);
        // factored form: the camera's t_x, t_y, f, k1, k2 for every observation of the chunk
        float ct0 = 0.f, ct1 = 0.f, cf = 0.f, ck1 = 0.f, ck2 = 0.f;
        if (FACT) {
            ct0 = (float)ct[18];
            ct1 = (float)ct[19];
            cf = (float)ct[21];
            ck1 = (float)ct[22];
            ck2 = (float)ct[23];
        }
        for (int s0 = b0; s0 < b1; s0 += 32 * U) {
            // s arrives in camera-major order (the point pass scattered it), so
            // every load of the batch is a coalesced stream
            bool in[U];
            float rx0[U], rx1[U], rx2[U], rz[U];  // R X and 1 / P_z
            T2 sv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int s = s0 + u * 32 + lane;
                in[u] = s < b1;
                if (in[u]) sv[u] = ldcg(sbuf + s);
                if (FACT) {
                    const float4 v = in[u] ? __ldcs((const float4 *)P.RXcm + s) : make_float4(0.f, 0.f, 0.f, 0.f);
                    rx0[u] = v.x;
                    rx1[u] = v.y;
                    rx2[u] = v.z;
                    rz[u] = v.w;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (in[u]) {
                    if (FACT) {
                        // y_t = D^T s = -(1/Pz) (g0, g1, p.g) with g = A s; accumulate
                        // y_t, RX x y_t, and p.s (d, r2, r2^2)
                        const float X0 = rx0[u], X1 = rx1[u], X2 = rx2[u];
                        const float s0v = (float)sv[u].x, s1v = (float)sv[u].y;
                        const float iz = rz[u];
                        const float x = -(X0 + ct0) * iz, y = -(X1 + ct1) * iz;
                        const float r2 = x * x + y * y;
                        const float d = 1.f + ck1 * r2 + ck2 * r2 * r2;
                        const float dd = 2.f * ck1 + 4.f * ck2 * r2;
                        const float a00 = cf * (d + dd * x * x), a01 = cf * dd * x * y, a11 = cf * (d + dd * y * y);
                        const float g0 = a00 * s0v + a01 * s1v, g1 = a01 * s0v + a11 * s1v;
                        const float y0 = -iz * g0, y1 = -iz * g1, y2 = x * y0 + y * y1;
                        acc[0] += (T)y0;
                        acc[1] += (T)y1;
                        acc[2] += (T)y2;
                        acc[3] += (T)(X1 * y2 - X2 * y1);
                        acc[4] += (T)(X2 * y0 - X0 * y2);
                        acc[5] += (T)(X0 * y1 - X1 * y0);
                        const float pss = x * s0v + y * s1v;
                        acc[6] += (T)(d * pss);
                        acc[7] += (T)(r2 * pss);
                        acc[8] += (T)(r2 * r2 * pss);
                    } else {
                        camera_acc_stored<T>(P, s0 + u * 32 + lane, (T)sv[u].x, (T)sv[u].y, acc);
                    }
                }
            }
        }
        T mine = T(0);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            T v = acc[a];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(full, v, d);
            if (FACT) acc[a] = v;  // every lane holds every sum
            else if (lane == a) mine = v;
        }
        if (FACT) {
            // Jc^T s of the chunk: rotation (R M)^T sum RX x y_t, translation
            // sum y_t, intrinsics (sum d p.s, f sum r2 p.s, f sum r2^2 p.s)
            const float Y0 = (float)acc[0], Y1 = (float)acc[1], Y2 = (float)acc[2];
            const float c0 = (float)acc[3], c1 = (float)acc[4], c2 = (float)acc[5];
            const float q0 = ct[0] * c0 + ct[3] * c1 + ct[6] * c2;  // R^T c
            const float q1 = ct[1] * c0 + ct[4] * c1 + ct[7] * c2;
            const float q2 = ct[2] * c0 + ct[5] * c1 + ct[8] * c2;
            const int a = lane < 3 ? lane : 0;
            const float yr = ct[9 + a] * q0 + ct[12 + a] * q1 + ct[15 + a] * q2;  // (M^T q)_a
            float mv = yr;
            if (lane == 3) mv = Y0;
            if (lane == 4) mv = Y1;
            if (lane == 5) mv = Y2;
            if (lane == 6) mv = (float)acc[6];
            if (lane == 7) mv = cf * (float)acc[7];
            if (lane == 8) mv = cf * (float)acc[8];
            mine = (T)mv;
        }
        if (lane < 9) cslot[(k - k0) * 9 + lane] = (double)mine;  // one conversion per lane
        int nk = 0;
        if (lane == 0) nk = atomicAdd(&next_chunk, 1);
        k = __shfl_sync(full, nk, 0);
    }
    __syncthreads();
    // finalise this CTA's cameras, three per warp (lanes 9s..9s+8 hold rows of
    // camera s): chunk sums added in chunk order
    double d1 = 0.0, d2 = 0.0, d3 = 0.0;
    const int sub = lane / 9, row = lane - 9 * sub;
    for (int c0 = cb + 3 * wid; c0 < ce; c0 += 3 * nwarp) {
        const int cam = c0 + sub;
        const bool act = lane < 27 && cam < ce;
        const int a = act ? row : 0;
        const int cm = act ? cam : c0;
        const int64_t vo = (int64_t)cm * kVec + a;
        // this lane's row of B~^-1 (right-hand side) or B~ (products): in the
        // factored form's standard iterations loaded before the chunk sums, so
        // that its latency overlaps them (109.9 -> 109.3 us per PCG iteration);
        // elsewhere loaded where it is used (the early load raised the
        // single-reduction instance's spills and slowed it, and the FP64 one)
        constexpr bool kEarly = FACT && MODE == CAM_ITER;
        const double *Mrow = (MODE == CAM_RHS ? P.Binv : P.Bd) + 81 * (int64_t)cm + a * 9;
        double brow[9];
#pragma unroll
        for (int b = 0; b < 9; ++b) brow[b] = (kEarly && act) ? __ldg(Mrow + b) : 0.0;
        double cs = 0.0;
        if (act)
            for (int k = P.cfirst[cm]; k < P.cfirst[cm + 1]; ++k) cs += cslot[(k - k0) * 9 + a];
        // a fixed camera has no Schur coupling (its Jacobian columns are zero; the
        // factored product forms Jc^T s from the geometry, so it is masked here)
        if (P.has_fixed && act && P.cam_fixed[cm]) cs = 0.0;
        double v1 = 0.0, v2 = 0.0, v3 = 0.0;
        if (MODE == CAM_RHS) {
            const double g = act ? P.v[9 * (int64_t)cm + a] - cs : 0.0;
            double z = 0.0;
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                const double gb = __shfl_sync(full, g, 9 * sub + b);
                if (act) z = fma(kEarly ? brow[b] : __ldg(Mrow + b), gb, z);
            }
            if (act) {
                stcg(P.g + vo, g);
                stcg(P.x + vo, 0.0);
                stcg(P.r + vo, g);
                stcg(P.z + vo, z);
                if (sizeof(T) == 4 && !FACT) stcg((float *)P.zT + vo, (float)z);
                v1 = g * g;
                v2 = g * z;
            }
            if (FACT) fact_row_store(P, (float *)P.zT, cm, act, z, sub, row, true);
        } else {
            double p = 0.0;
            if (act) {
                if (MODE == CAM_MATVEC) p = P.p[vo];
                else if (MODE == CAM_SR) p = ldcg(P.z + vo);
                else p = first ? ldcg(P.z + vo) : fma(beta, ldcg(p_prev + vo), ldcg(P.z + vo));
            }
            double bp = 0.0;
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                const double pb = __shfl_sync(full, p, 9 * sub + b);
                if (act) bp = fma(kEarly ? brow[b] : __ldg(Mrow + b), pb, bp);
            }
            const double q = act ? bp - cs : 0.0;
            if (act) {
                stcg(P.q + vo, q);
                if (MODE == CAM_ITER) {
                    stcg(p_cur + vo, p);
                    if (pT_cur && !FACT) stcg(pT_cur + vo, (T)p);
                }
                if (MODE == CAM_SR) {
                    const double rv = ldcg(P.r + vo);
                    v1 = rv * rv;
                    v2 = rv * p;
                    v3 = q * p;
                } else {
                    v1 = p * q;
                }
            }
            if (FACT && MODE == CAM_ITER && pT_cur) fact_row_store(P, (float *)pT_cur, cm, act, p, sub, row, false);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            v1 += __shfl_xor_sync(full, v1, d);
            v2 += __shfl_xor_sync(full, v2, d);
            if (MODE == CAM_SR) v3 += __shfl_xor_sync(full, v3, d);
        }
        d1 += v1;
        d2 += v2;
        d3 += v3;
    }
    if constexpr (MODE == CAM_SR) {
        const double3 t = cta_sum3(lane == 0 ? d1 : 0.0, lane == 0 ? d2 : 0.0, lane == 0 ? d3 : 0.0, false, sb);
        *third = t.z;
        return make_double2(t.x, t.y);
    }
    // CTA partials in a fixed order (warp w's cameras, then a tree over warps);
    // d1, d2 are already warp-uniform, so no per-warp shuffle tree is needed
    return cta_sum2(lane == 0 ? d1 : 0.0, lane == 0 ? d2 : 0.0, false, sb);
}

// Search direction into shared memory (dense nc x 9, in T): p = z + beta p_prev
// (p = z on the first iteration), or the given FP64 p (src_given).  The FP32
// form builds it from float copies of z and p_prev with float4 loads; the FP64
// form from the FP64 vectors, as the camera pass does.
// Factored form: the camera rows ([nc][kRow] floats) instead: row(z) + beta
// row(p_prev) from the float row copies, or the rows of the given FP64 p.
template <typename T, bool FACT>
__device__ void stage_p(const Prob &P, T *ps, const double *p_prev, const T *pT_prev, double beta, bool first,
                        const double *src_given) {
    if constexpr (FACT) {
        float4 *dst = (float4 *)ps;
        if (!src_given) {
            const float4 *z4 = (const float4 *)P.zT, *p4 = (const float4 *)pT_prev;
            const float fb = (float)beta;
            const int nq = P.nc * (kRow / 4);  // float4 per camera row
            for (int e = threadIdx.x; e < nq; e += blockDim.x) {
                const float4 zv = __ldcg(z4 + e);
                float4 v = zv;
                if (!first) {
                    const float4 pv = __ldcg(p4 + e);
                    v = make_float4(fmaf(fb, pv.x, zv.x), fmaf(fb, pv.y, zv.y), fmaf(fb, pv.z, zv.z),
                                    fmaf(fb, pv.w, zv.w));
                }
                dst[e] = v;
            }
        } else {
            for (int cam = threadIdx.x; cam < P.nc; cam += blockDim.x) {
                float v[9], r[kRow];
#pragma unroll
                for (int j = 0; j < 9; ++j) v[j] = (float)src_given[(int64_t)cam * kVec + j];
                fact_row((const float *)P.camtab + (int64_t)cam * kCamTab, v, true, r);
#pragma unroll
                for (int i = 0; i < kRow / 4; ++i)
                    dst[(kRow / 4) * cam + i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
            }
        }
        __syncthreads();
        return;
    }
    const int total = P.nc * 9;
    if (sizeof(T) == 4 && !src_given) {
        const float4 *z4 = (const float4 *)P.zT, *p4 = (const float4 *)pT_prev;
        const float fb = (float)beta;
        const int nq = P.nc * (kVec / 4);  // float4 per camera row: 3 (9 values + padding)
        for (int e = threadIdx.x; e < nq; e += blockDim.x) {
            const int cam = e / 3, part = e - cam * 3;
            const float4 zv = __ldcg(z4 + e);
            float4 v = zv;
            if (!first) {
                const float4 pv = __ldcg(p4 + e);
                v = make_float4(fmaf(fb, pv.x, zv.x), fmaf(fb, pv.y, zv.y), fmaf(fb, pv.z, zv.z), fmaf(fb, pv.w, zv.w));
            }
            float *dst = (float *)ps + cam * 9 + part * 4;
            dst[0] = v.x;
            if (part < 2) {
                dst[1] = v.y;
                dst[2] = v.z;
                dst[3] = v.w;
            }
        }
        __syncthreads();
        return;
    }
    constexpr int U = 4;
    for (int e0 = threadIdx.x; e0 < total; e0 += blockDim.x * U) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = 0.0;
            if (e < total) {
                const int cam = e / 9, a = e - cam * 9;
                const int64_t vo = (int64_t)cam * kVec + a;
                if (src_given) v[u] = src_given[vo];
                else v[u] = first ? ldcg(P.z + vo) : fma(beta, ldcg(p_prev + vo), ldcg(P.z + vo));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < total) ps[e] = (T)v[u];
        }
    }
    __syncthreads();
}

// CTA-wide sums of two doubles in a fixed tree order; every thread gets the
// result.  With warp_data (warp-uniform) the warp first reduces its lanes by a
// shuffle tree; without it lane 0's value is taken as the warp's sum, so warps
// with nothing (or a single value) skip the tree: GB300's FP64 pipe takes 16
// cycles per warp instruction.  Warp 0 then adds the per-warp sums.
__device__ __forceinline__ double2 cta_sum2(double x, double y, bool warp_data, double *sb) {
    __shared__ double2 s_out2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (warp_data) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
    }
    __syncthreads();
    if (lane == 0) {
        sb[wid] = x;  // lane 0 holds the warp's sum (or its only value)
        sb[32 + wid] = y;
    }
    __syncthreads();
    if (wid == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        double sx = in ? sb[lane] : 0.0, sy = in ? sb[32 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_down_sync(0xffffffffu, sx, o);
            sy += __shfl_down_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) s_out2 = make_double2(sx, sy);
    }
    __syncthreads();
    return s_out2;
}


// Two sums of n per-CTA partials (n <= blockDim.x: one load per thread, then
// shuffle trees only in the warps that hold partials); every thread of every
// CTA gets the same values.
__device__ __forceinline__ double2 sum_parts2(const double *a, const double *b, int n, double *sb) {
    double x = 0.0, y = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        x += ldcg(a + i);
        y += b ? ldcg(b + i) : 0.0;
    }
    return cta_sum2(x, y, (int)(threadIdx.x & ~31u) < n, sb);
}

__device__ __forceinline__ double sum_parts(const double *parts, int n, double *sb) {
    return sum_parts2(parts, nullptr, n, sb).x;
}

// Three-value forms of cta_sum2 / sum_parts2 (the single-reduction PCG); sb
// holds 96 doubles.
__device__ __forceinline__ double3 cta_sum3(double x, double y, double z, bool warp_data, double *sb) {
    __shared__ double3 s_out3;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (warp_data) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
            z += __shfl_down_sync(0xffffffffu, z, o);
        }
    }
    __syncthreads();
    if (lane == 0) {
        sb[wid] = x;
        sb[32 + wid] = y;
        sb[64 + wid] = z;
    }
    __syncthreads();
    if (wid == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        double sx = in ? sb[lane] : 0.0, sy = in ? sb[32 + lane] : 0.0, sz = in ? sb[64 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_down_sync(0xffffffffu, sx, o);
            sy += __shfl_down_sync(0xffffffffu, sy, o);
            sz += __shfl_down_sync(0xffffffffu, sz, o);
        }
        if (lane == 0) s_out3 = make_double3(sx, sy, sz);
    }
    __syncthreads();
    return s_out3;
}

__device__ __forceinline__ double3 sum_parts3(const double *a, const double *b, const double *c, int n, double *sb) {
    double x = 0.0, y = 0.0, z = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        x += ldcg(a + i);
        y += ldcg(b + i);
        z += ldcg(c + i);
    }
    return cta_sum3(x, y, z, (int)(threadIdx.x & ~31u) < n, sb);
}

// ---------------------------------------------------------------------------
// persistent PCG kernel (cooperative launch, one CTA per SM for the whole solve)
// ---------------------------------------------------------------------------
// JS: the camera pass reads the stored camera-major Jacobian (always in FP64;
// in FP32-mixed when the Jacobian comes from dual numbers).
// STG: the staged point pass (factored form only, a separate instantiation so
// that its code does not weigh on the direct pass's registers).
// SR: the single-reduction recurrence (mba_pcg_variant), also its own instance.
template <typename T, bool JS, bool STG, bool SR>
__global__ void __launch_bounds__(PcgBlock<T>::value, 1)
    pcg_kernel(Prob P, int mode, int max_iter, double tol, long long spin, int forcing) {
    using T2 = typename V2<T>::type;
    constexpr bool FACT = sizeof(T) == 4 && !JS;  // FP32-mixed, analytic Jacobian: the factored form
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double sb[96];
    DevState *st = P.st;
    if (st->done || st->blockfail) return;  // a failed damping: the LM loop rejects this iteration
    // forcing sequence: the first solve's right-hand side norm as it was before
    // this launch, read before the first grid barrier (block 0 writes it after
    // the last one)
    __shared__ double s_g0;
    if (threadIdx.x == 0) s_g0 = forcing ? st->g0 : 0.0;
    uint32_t epoch = 0;
    const int G = gridDim.x;
    const int nwarp = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *pT = (T *)P.pT;
    T2 *sbuf = (T2 *)P.sbuf;
    double *part_rho = P.red, *part_rr = P.red + G, *part_pq = P.red + 2 * G;
    const int ncw = (P.nc + 2) / 3;  // warps of camera-row work (3 cameras x 9 rows per warp)
    const int my_sub = lane / 9, row = lane % 9;
    const unsigned full = 0xffffffffu;
    T *ps = P.pcg_use_ps ? (T *)smem_raw : nullptr;
    double *cslot = (double *)(smem_raw + P.pcg_ps_bytes);
    bool ok = true;
    auto barrier = [&]() -> bool { return grid_barrier(st, epoch, spin); };
    // staged point pass (factored form): stage barriers, use counters, and the
    // drain that waits for copies still in flight before the CTA leaves
    __shared__ __align__(8) uint64_t s_full[kMaxStages], s_empty[kMaxStages];
    __shared__ StageOrg s_org[kMaxStages];
    const int S = (FACT && STG) ? P.pcg_stages : 0;
    const uint32_t Su = S > 0 ? (uint32_t)S : 1u;
    unsigned char *stages = smem_raw + P.pcg_stage_off;
    const int my_nt = (S && P.n_tiles > (int)blockIdx.x) ? (P.n_tiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    uint32_t use = 0, issued = 0;
    if (STG && S) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < S; ++i) {
                mbar_init(s_full + i, 1);
                mbar_init(s_empty + i, (uint32_t)(nwarp - 1));
            }
            mbar_init_fence();
        }
        __syncthreads();
    }
    // the producer warp's first lane waits for the copies it issued beyond the
    // last consumed use before the CTA leaves
    auto drain = [&]() {
        if (STG && S && threadIdx.x == (unsigned)(nwarp - 1) * 32)
            for (uint32_t u = use; u < issued; ++u)
                if (!mbar_wait(s_full + u % Su, (u / Su) & 1u, kStageSpin)) {
                    atomicCAS(&st->err, 0, (int)MBA_ERR_TIMEOUT);
                    break;
                }
    };
    // the point pass of one product; rows: the search rows in global memory
    // (read where they are not in shared memory)
    auto point_pass_iter = [&](const T *rows) -> bool {
        if constexpr (FACT && STG) {
            if (S)
                return point_pass_fact_staged(P, (const float *)ps, (const float *)rows, (float2 *)sbuf, stages,
                                              s_full, s_empty, s_org, S, my_nt, use, issued);
        }
        point_pass_any<T, false, FACT>(P, ps, rows, sbuf);
        return true;
    };
    // owner phase: p = z + beta p_prev written in FP64 and, for the gathers, as
    // T (or, in the factored form, as the camera's row)
    auto phase_p = [&](const double *p_prev, double *p_cur, double beta, bool first, const double *given) {
        for (int w = blockIdx.x * nwarp + wid; w < ncw; w += G * nwarp) {
            const int cam = w * 3 + my_sub;
            const bool act = lane < 27 && cam < P.nc;
            double pn = 0.0;
            if (act) {
                const int64_t vo = (int64_t)cam * kVec + row;
                pn = given ? given[vo] : (first ? ldcg(P.z + vo) : fma(beta, ldcg(p_prev + vo), ldcg(P.z + vo)));
                if (!given) stcg(p_cur + vo, pn);
                if (!FACT) stcg(pT + vo, (T)pn);
            }
            if (FACT) fact_row_store(P, (float *)pT, act ? cam : 0, act, pn, my_sub, row, true);
        }
    };

    if (mode == PCG_MATVEC) {
        // p given in P.p (FP64): q = B~ p - E C~^-1 E^T p
        if (ps) {
            stage_p<T, FACT>(P, ps, nullptr, nullptr, 0.0, true, P.p);
        } else {
            phase_p(nullptr, nullptr, 0.0, true, P.p);
            if (!(ok = barrier())) return;
        }
        const bool pok = point_pass_iter(pT);
        if (pok && barrier()) camera_pass<T, CAM_MATVEC, JS>(P, sbuf, nullptr, nullptr, nullptr, 0.0, true, cslot, sb);
        drain();
        return;
    }

    // ---- right-hand side g = v - E C~^-1 w (Eq. 3), x = 0, r = g, z = B~^-1 g ----
    point_pass_any<T, true, FACT>(P, nullptr, nullptr, sbuf);
    ok = barrier();
    if (ok) {
        const double2 d = camera_pass<T, CAM_RHS, JS>(P, sbuf, nullptr, nullptr, nullptr, 0.0, true, cslot, sb);
        if (mode == PCG_RHS_ONLY) return;
        if (threadIdx.x == 0) {
            stcg(part_rr + blockIdx.x, d.x);
            stcg(part_rho + blockIdx.x, d.y);
        }
        ok = barrier();
    }

    if constexpr (SR) {
        // Single-reduction PCG (Chronopoulos-Gear form; the oracle's
        // pcg_single_reduction).  Step n: the point pass forms s~ for u_n,
        // barrier, the camera pass gives w_n = S~ u_n at each camera's owner and
        // the partials of r.r, r.u and w.u, barrier, then every CTA derives
        // alpha and beta from the three sums and the owners update p, s, x, r
        // and u = B~^-1 r and write u's rows, which a third barrier publishes
        // to the next point pass.  Three barriers and one reduction per step
        // (the standard loop: three barriers and two reductions with the rows
        // in shared memory, four barriers otherwise).
        // Not kept: a two-barrier form in which every CTA formed u's rows from
        // the recurrence u_{n+1} = u_n - alpha B~^-1 s_n in FP32.  As |u| falls
        // over the solve, that subtraction cancels and the FP32 rounding of the
        // earlier, larger terms dominates: 1e-3 relative error in the step after
        // 10 PCG steps and 0.03 to 0.15 after 30, against 1.5e-5 for the rows
        // written by the owners.
        __shared__ double s_alpha, s_beta, s_r0, s_rn, s_stop2, s_gprev, s_aprev;
        __shared__ int s_go;
        // where the point pass finds u's rows when they are not in shared memory
        const T *rows_u = sizeof(T) == 8 ? (const T *)P.z : (const T *)P.zT;
        int n = 0;
        while (ok && (n == 0 || n < max_iter)) {
            if (ps) stage_p<T, FACT>(P, ps, nullptr, nullptr, 0.0, true, nullptr);
            if (!(ok = point_pass_iter(rows_u))) break;
            if (!(ok = barrier())) break;
            {
                double wu = 0.0;
                const double2 d =
                    camera_pass<T, CAM_SR, JS>(P, sbuf, nullptr, nullptr, nullptr, 0.0, false, cslot, sb, &wu);
                if (threadIdx.x == 0) {
                    stcg(part_rr + blockIdx.x, d.x);
                    stcg(part_rho + blockIdx.x, d.y);
                    stcg(part_pq + blockIdx.x, wu);
                }
            }
            if (!(ok = barrier())) break;
            const double3 sums = sum_parts3(part_rr, part_rho, part_pq, G, sb);
            if (threadIdx.x == 0) {
                // sums: r.r, gamma = r.u, delta = w.u
                bool go;
                if (n == 0) {
                    const double r0 = sqrt(sums.x);
                    double t = tol;
                    if (forcing) {  // eta = min(0.1, sqrt(|g| / |g_first|)), |g_first| = r0 in the first solve
                        const double g0 = s_g0;
                        t = fmax(t, fmin(0.1, sqrt(r0 / (g0 > 0.0 ? g0 : r0))));
                    }
                    s_r0 = r0;
                    s_stop2 = (t * r0) * (t * r0);
                    go = r0 > 0.0;
                } else {
                    go = !(sums.x <= s_stop2);
                }
                s_rn = sqrt(sums.x);
                go = go && isfinite(sums.y);
                const double beta = n == 0 ? 0.0 : sums.y / s_gprev;
                const double den = n == 0 ? sums.z : sums.z - beta * sums.y / s_aprev;  // p.S p
                go = go && den > 0.0 && isfinite(den);
                const double alpha = go ? sums.y / den : 0.0;
                s_gprev = sums.y;
                s_aprev = alpha;
                s_alpha = alpha;
                s_beta = beta;
                s_go = go ? 1 : 0;
            }
            __syncthreads();
            if (!s_go) break;
            const double alpha = s_alpha, beta = s_beta;
            // p = u + beta p, s = w + beta s (s in the free second direction buffer),
            // x += alpha p, r -= alpha s, u = B~^-1 r over this CTA's own cameras
            const bool last = n + 1 >= max_iter;  // the step cap ends the solve after this update
            {
                double *sv = P.p2;
                double rr = 0.0;  // |r|^2 after the update, taken on the last step only
                const int cb = P.cta_cam[blockIdx.x], ce = P.cta_cam[blockIdx.x + 1];
                for (int c0 = cb + 3 * wid; c0 < ce; c0 += 3 * nwarp) {
                    const int cam = c0 + my_sub;
                    const bool act = lane < 27 && cam < ce;
                    const int64_t vo = (int64_t)(act ? cam : c0) * kVec + row;
                    double rv = 0.0;
                    if (act) {
                        const double u = ldcg(P.z + vo), w = ldcg(P.q + vo);
                        const double pn = n == 0 ? u : fma(beta, ldcg(P.p + vo), u);
                        const double sn = n == 0 ? w : fma(beta, ldcg(sv + vo), w);
                        stcg(P.p + vo, pn);
                        stcg(sv + vo, sn);
                        stcg(P.x + vo, fma(alpha, pn, ldcg(P.x + vo)));
                        rv = fma(-alpha, sn, ldcg(P.r + vo));
                        stcg(P.r + vo, rv);
                        rr = fma(rv, rv, rr);
                    }
                    double z = 0.0;
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
                        const double rc = __shfl_sync(full, rv, my_sub * 9 + c);
                        if (act) z = fma(__ldg(P.Binv + 81 * (int64_t)cam + row * 9 + c), rc, z);
                    }
                    if (FACT) fact_row_store(P, (float *)P.zT, act ? cam : c0, act, z, my_sub, row, true);
                    if (act) {
                        stcg(P.z + vo, z);
                        if (sizeof(T) == 4 && !FACT) stcg((float *)P.zT + vo, (float)z);
                    }
                }
                if (last) {
                    // the residual norm the solve reports, in its own partials (the
                    // step's sums may still be read by other CTAs)
                    const double2 t = cta_sum2(rr, 0.0, true, sb);
                    if (threadIdx.x == 0) stcg(P.red + 3 * G + blockIdx.x, t.x);
                }
            }
            ++n;
            if (last) {
                if (!(ok = barrier())) break;
                const double rrn = sum_parts(P.red + 3 * G, G, sb);
                if (threadIdx.x == 0) s_rn = sqrt(rrn);
                __syncthreads();
                break;
            }
            if (!(ok = barrier())) break;
        }
        drain();
        if (!ok) atomicCAS(&st->err, 0, (int)MBA_ERR_TIMEOUT);
        if (ok && blockIdx.x == 0 && threadIdx.x == 0) {
            st->pcg_iters = n;
            st->pcg_rel_res = s_r0 > 0.0 ? s_rn / s_r0 : 0.0;
            if (forcing && !(s_g0 > 0.0)) st->g0 = s_r0;
        }
        return;
    }

    // The scalar recurrences (r0, rho, alpha, beta, the stopping test) run in
    // thread 0 alone and are broadcast through shared memory: on this GPU each
    // warp-wide FP64 instruction holds the SM's FP64 pipe for 16 cycles and a
    // division or square root is a chain of about ten of them, so evaluating
    // them redundantly in all 1024 threads would stall every CTA for microseconds.
    // Thread 0's state (r0, rho, |r|, the stopping threshold) also lives in
    // shared memory, so that no register stays reserved for it through the loop.
    __shared__ double s_alpha, s_beta, s_r0, s_rho, s_rn, s_stop;
    __shared__ int s_go;
    int n = 0;
    if (ok) {
        const double2 s0 = sum_parts2(part_rr, part_rho, G, sb);
        if (threadIdx.x == 0) {
            const double r0 = sqrt(s0.x);
            double t = tol;
            if (forcing) {  // eta = min(0.1, sqrt(|g| / |g_first|)), |g_first| = r0 in the first solve
                const double g0 = s_g0;
                t = fmax(t, fmin(0.1, sqrt(r0 / (g0 > 0.0 ? g0 : r0))));
            }
            s_r0 = r0;
            s_rho = s0.y;
            s_rn = r0;
            s_stop = t * r0;
            s_go = (r0 > 0.0 && isfinite(s0.y)) ? 1 : 0;
            s_beta = 0.0;
        }
        __syncthreads();
    }
    if (ok && s_go) {
        for (;;) {
            const double beta = s_beta;
            double *p_cur = (n & 1) ? P.p2 : P.p;
            const double *p_prev = (n & 1) ? P.p : P.p2;
            T *pT_cur = (n & 1) ? (T *)P.pT2 : pT;
            const T *pT_prev = (n & 1) ? pT : (T *)P.pT2;
            if (ps) {
                stage_p<T, FACT>(P, ps, p_prev, pT_prev, beta, n == 0, nullptr);
            } else {
                phase_p(p_prev, p_cur, beta, n == 0, nullptr);
                if (!(ok = barrier())) break;
            }
            if (!(ok = point_pass_iter(pT))) break;
            if (!(ok = barrier())) break;
            {
                const double2 d = camera_pass<T, CAM_ITER, JS>(P, sbuf, p_prev, p_cur,
                                                               (sizeof(T) == 4 && ps) ? pT_cur : nullptr,
                                                           beta, n == 0, cslot, sb);
                if (threadIdx.x == 0) stcg(part_pq + blockIdx.x, d.x);
            }
            if (!(ok = barrier())) break;
            const double pq = sum_parts(part_pq, G, sb);
            if (threadIdx.x == 0) {
                const bool go = (pq > 0.0) && isfinite(pq);
                s_go = go ? 1 : 0;
                s_alpha = go ? s_rho / pq : 0.0;
            }
            __syncthreads();
            if (!s_go) break;
            const double alpha = s_alpha;
            // x += alpha p; r -= alpha q; z = B~^-1 r; partial r.r and r.z, over this
            // CTA's own cameras (three per warp)
            {
                double rr = 0.0, rz = 0.0;
                const int cb = P.cta_cam[blockIdx.x], ce = P.cta_cam[blockIdx.x + 1];
                for (int c0 = cb + 3 * wid; c0 < ce; c0 += 3 * nwarp) {
                    const int cam = c0 + my_sub;
                    const bool act = lane < 27 && cam < ce;
                    const int64_t vo = (int64_t)(act ? cam : c0) * kVec + row;
                    // this lane's row of B~^-1, loaded beside (not after) the r update
                    double bi[9];
#pragma unroll
                    for (int c = 0; c < 9; ++c) bi[c] = act ? __ldg(P.Binv + 81 * (int64_t)cam + row * 9 + c) : 0.0;
                    double rv = 0.0;
                    if (act) {
                        stcg(P.x + vo, fma(alpha, ldcg(p_cur + vo), ldcg(P.x + vo)));
                        rv = fma(-alpha, ldcg(P.q + vo), ldcg(P.r + vo));
                        stcg(P.r + vo, rv);
                    }
                    double z = 0.0;
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
                        const double rc = __shfl_sync(full, rv, my_sub * 9 + c);
                        z = fma(bi[c], rc, z);
                    }
                    if (FACT) fact_row_store(P, (float *)P.zT, act ? cam : c0, act, z, my_sub, row, true);
                    if (act) {
                        stcg(P.z + vo, z);
                        if (sizeof(T) == 4 && !FACT) stcg((float *)P.zT + vo, (float)z);
                        rr += rv * rv;
                        rz += rv * z;
                    }
                }
                const bool has = cb + 3 * wid < ce;
                const double2 sr = cta_sum2(rr, rz, has, sb);
                if (threadIdx.x == 0) {
                    stcg(part_rr + blockIdx.x, sr.x);
                    stcg(part_rho + blockIdx.x, sr.y);
                }
            }
            if (!(ok = barrier())) break;
            ++n;
            const double2 sums = sum_parts2(part_rho, part_rr, G, sb);
            if (threadIdx.x == 0) {
                const double rho_prev = s_rho, rho = sums.x, rn = sqrt(sums.y);
                s_rho = rho;
                s_rn = rn;
                const bool go = !(rn <= s_stop || n >= max_iter) && isfinite(rho);
                s_go = go ? 1 : 0;
                s_beta = go ? rho / rho_prev : 0.0;
            }
            __syncthreads();
            if (!s_go) break;
        }
    }
    drain();
    if (!ok) atomicCAS(&st->err, 0, (int)MBA_ERR_TIMEOUT);
    if (ok && blockIdx.x == 0 && threadIdx.x == 0) {
        st->pcg_iters = n;
        st->pcg_rel_res = s_r0 > 0.0 ? s_rn / s_r0 : 0.0;
        if (forcing && !(s_g0 > 0.0)) st->g0 = s_r0;
    }
}

// ---------------------------------------------------------------------------
// back-substitution dp_j = C~_j^-1 (w_j - sum_k Jp~_k^T Jc~_k dc_i(k)) (Eq. 4),
// candidate points, and the model decrease sum_k (-e~_k.d_k - |d_k|^2/2)
// with d_k = Jc~_k dc + Jp~_k dp.
// ---------------------------------------------------------------------------
// Per observation: t = Jc dc (sqrt(W)-scaled in the stored form, unscaled in
// FACT) and the point-side Jacobian (Jp~, or W Jp in FACT), so that
// u = jp^T t is this observation's term of Jp~^T Jc~ dc.
template <typename T, bool FACT>
__device__ __forceinline__ void backsub_obs(const Prob &P, int64_t o, int cam, T *t, T *jp) {
    const int64_t npad = P.npad;
    if constexpr (FACT) {
        float r[kRow];
        gather_row(nullptr, (const float *)P.pT, cam, r);
        fact_jc_v(__ldcs(P.PXpm + o), __ldcs(P.PXpm + npad + o), __ldcs(P.PXpm + 2 * npad + o), r, t);
#pragma unroll
        for (int k = 0; k < 6; ++k) jp[k] = __ldcs(P.Jph + k * npad + o);
    } else {
        T Jc[18];
        load_jac_stream((const T *)P.J, npad, o, Jc, jp);
        const double *xc = P.x + (int64_t)cam * kVec;
        t[0] = t[1] = T(0);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const T xa = (T)xc[a];
            t[0] += Jc[a] * xa;
            t[1] += Jc[9 + a] * xa;
        }
    }
}
// Model-decrease term of one observation given its point step: d~ = J~_k (dc, dp),
// -e~.d~ - |d~|^2 / 2 (FACT: d~ = sqrt(W) t + (W Jp) dp / sqrt(W)).
template <typename T, bool FACT>
__device__ __forceinline__ double backsub_dec(const Prob &P, int64_t o, const T *t, const T *jp, const T *dp) {
    T d0 = jp[0] * dp[0] + jp[1] * dp[1] + jp[2] * dp[2];
    T d1 = jp[3] * dp[0] + jp[4] * dp[1] + jp[5] * dp[2];
    if constexpr (FACT) {
        const float sw = P.swpm ? __ldg(P.swpm + o) : 1.f, isw = 1.f / sw;
        d0 = sw * t[0] + isw * d0;
        d1 = sw * t[1] + isw * d1;
    } else {
        d0 += t[0];
        d1 += t[1];
    }
    const T *res = (const T *)P.res;
    const double e0 = (double)__ldcs(res + o), e1 = (double)__ldcs(res + P.npad + o);
    const double dd0 = (double)d0, dd1 = (double)d1;
    return -(e0 * dd0 + e1 * dd1) - 0.5 * (dd0 * dd0 + dd1 * dd1);
}
// The point step dp_j = C~_j^-1 (w_j - a), its FP64 copy and the candidate point.
template <typename T>
__device__ __forceinline__ void backsub_point(const Prob &P, int pt, const T *a, T *dp) {
    const T t0 = (T)P.w[3 * (int64_t)pt] - a[0], t1 = (T)P.w[3 * (int64_t)pt + 1] - a[1],
            t2 = (T)P.w[3 * (int64_t)pt + 2] - a[2];
    sym3_apply((const T *)P.Cinv + 6 * (int64_t)pt, t0, t1, t2, dp);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        P.dp[3 * (int64_t)pt + k] = (double)dp[k];
        P.pts_new[3 * (int64_t)pt + k] = P.pts[3 * (int64_t)pt + k] + (double)dp[k];
    }
}

// ---------------------------------------------------------------------------
// back-substitution dp_j = C~_j^-1 (w_j - sum_k Jp~_k^T Jc~_k dc_i(k)) (Eq. 4),
// candidate points, and the model decrease sum_k (-e~_k.d_k - |d_k|^2/2)
// with d_k = Jc~_k dc + Jp~_k dp, in one sweep over point-major warp chunks:
// a segmented scan gives each point's sum, its last lane forms dp and the
// point's lanes take it by a shuffle.  FACT (FP32-mixed analytic): t = Jc dc
// from the camera rows of dc (fact_rows_kernel, into the free search-direction
// buffer) and (px, py, 1/Pz).
// ---------------------------------------------------------------------------
template <typename T, bool FACT>
__global__ void __launch_bounds__(kBlock) backsub_kernel(Prob P, double *partial) {
    __shared__ double sb[kWarps];
    if (P.st->done) return;
    const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;
    double ldec = 0.0;
    for (int w = blockIdx.x * nwarp + (threadIdx.x >> 5); w < P.n_wchunks; w += gridDim.x * nwarp) {
        const int2 c0 = P.wchunk[w], c1 = P.wchunk[w + 1];
        const int o0 = c0.y, m = c1.y - c0.y;
        if (m <= 32) {
            const bool act = lane < m;
            const int64_t o = (int64_t)o0 + (act ? lane : 0);
            const int npts = c1.x - c0.x;
            const int rs = lane < npts ? __ldg(P.pt_ptr + c0.x + lane) - o0 : 32;
            const unsigned starts = __reduce_or_sync(full, rs < 32 ? (1u << rs) : 0u);
            const int pt = act ? c0.x + __popc(starts & (0xffffffffu >> (31 - lane))) - 1 : -1 - lane;
            T t[2] = {T(0), T(0)}, jp[6], u[3];
#pragma unroll
            for (int k = 0; k < 6; ++k) jp[k] = T(0);
            if (act) backsub_obs<T, FACT>(P, o, __ldg(P.pm_cam + o), t, jp);
            u[0] = jp[0] * t[0] + jp[3] * t[1];
            u[1] = jp[1] * t[0] + jp[4] * t[1];
            u[2] = jp[2] * t[0] + jp[5] * t[1];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int kp = __shfl_up_sync(full, pt, d);
                const T v0 = __shfl_up_sync(full, u[0], d), v1 = __shfl_up_sync(full, u[1], d),
                        v2 = __shfl_up_sync(full, u[2], d);
                if (lane >= d && kp == pt) {
                    u[0] += v0;
                    u[1] += v1;
                    u[2] += v2;
                }
            }
            const int nxt = __shfl_down_sync(full, pt, 1);
            const bool tail = act && (lane == m - 1 || nxt != pt);
            T dp[3] = {T(0), T(0), T(0)};
            if (tail) backsub_point<T>(P, pt, u, dp);
            const unsigned tails = __ballot_sync(full, tail);
            const unsigned mine = tails & (0xffffffffu << lane);
            const int src = mine ? __ffs(mine) - 1 : lane;
            T dq[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) dq[k] = __shfl_sync(full, dp[k], src);
            if (act) ldec += backsub_dec<T, FACT>(P, o, t, jp, dq);
        } else {
            // one point with a long track: the sum over 32-observation slices, then
            // a second sweep for the model decrease
            const int pt = c0.x;
            T a[3] = {T(0), T(0), T(0)};
            for (int base = 0; base < m; base += 32) {
                if (base + lane < m) {
                    const int64_t o = (int64_t)o0 + base + lane;
                    T t[2], jp[6];
                    backsub_obs<T, FACT>(P, o, __ldg(P.pm_cam + o), t, jp);
#pragma unroll
                    for (int k = 0; k < 3; ++k) a[k] += jp[k] * t[0] + jp[3 + k] * t[1];
                }
            }
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) a[k] += __shfl_xor_sync(full, a[k], d);
            T dp[3] = {T(0), T(0), T(0)};
            if (lane == 0) backsub_point<T>(P, pt, a, dp);
#pragma unroll
            for (int k = 0; k < 3; ++k) dp[k] = __shfl_sync(full, dp[k], 0);
            for (int base = 0; base < m; base += 32) {
                if (base + lane < m) {
                    const int64_t o = (int64_t)o0 + base + lane;
                    T t[2], jp[6];
                    backsub_obs<T, FACT>(P, o, __ldg(P.pm_cam + o), t, jp);
                    ldec += backsub_dec<T, FACT>(P, o, t, jp, dp);
                }
            }
        }
    }
    const double s = block_sum(ldec, sb);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Camera rows (with the constants) of the PCG solution dc, for the factored
// back-substitution; one thread per camera.
__global__ void fact_rows_kernel(Prob P, const double *__restrict__ x, float *__restrict__ rows) {
    if (P.st->done) return;
    for (int cam = blockIdx.x * blockDim.x + threadIdx.x; cam < P.nc; cam += gridDim.x * blockDim.x) {
        float v[9], r[kRow];
#pragma unroll
        for (int j = 0; j < 9; ++j) v[j] = (float)x[(int64_t)cam * kVec + j];
        fact_row((const float *)P.camtab + (int64_t)cam * kCamTab, v, true, r);
        float4 *dst = (float4 *)(rows + (int64_t)cam * kRow);
#pragma unroll
        for (int i = 0; i < kRow / 4; ++i) dst[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
    }
}

__global__ void cams_new_kernel(Prob P) {
    if (P.st->done) return;
    const int64_t total = (int64_t)P.nc * 9;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / 9, a = t % 9;
        P.cams_new[t] = P.cams[t] + P.x[i * kVec + a];
    }
}

__global__ void ldec_final_kernel(const double *partial, int nb, DevState *st) {
    __shared__ double sb[kWarps];
    if (st->done) return;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    const double s = block_sum(acc, sb);
    if (threadIdx.x == 0) st->model_dec = s;
}


}  // namespace

cudaError_t launch_damp(const Prob &P, int damping, int precond, const int32_t *cfirst, cudaStream_t s) {
    damp_cameras_kernel<<<(P.nc + kDampWarps - 1) / kDampWarps, 32 * kDampWarps, 0, s>>>(P, damping);
    const int64_t nb = (P.np + kBlock - 1) / kBlock;
    const unsigned g = (unsigned)(nb > 152 * 16 ? 152 * 16 : nb);
    if (P.fp32) damp_points_kernel<float><<<g, kBlock, 0, s>>>(P, damping);
    else damp_points_kernel<double><<<g, kBlock, 0, s>>>(P, damping);
    if (precond == MBA_PRECOND_SCHUR_JACOBI) {
        const unsigned gc = (unsigned)(P.n_cchunks < 152 * 4 ? (P.n_cchunks > 0 ? P.n_cchunks : 1) : 152 * 4);
        if (P.fp32) {
            if (P.autodiff) sj_camera_kernel<float, true><<<gc, kBlock, 0, s>>>(P);
            else sj_camera_kernel<float, false><<<gc, kBlock, 0, s>>>(P);
        } else {
            if (P.autodiff) sj_camera_kernel<double, true><<<gc, kBlock, 0, s>>>(P);
            else sj_camera_kernel<double, false><<<gc, kBlock, 0, s>>>(P);
        }
        sj_finalize_kernel<<<(P.nc + kDampWarps - 1) / kDampWarps, 32 * kDampWarps, 0, s>>>(P, cfirst);
    }
    return cudaGetLastError();
}

// Shared-memory plan: the camera-pass chunk slots of the busiest CTA, plus the
// search direction (nc x 9) when it also fits; otherwise the point pass
// gathers p from global memory and an extra barrier is needed.
void plan_pcg_smem(Prob &P) {
    const int w = P.fp32 ? 4 : 8;
    const int per_cam = P.fact ? kRow : 9;  // the factored form stages a kRow-float row per camera
    const int64_t budget = 227 * 1024 - 12 * 1024;
    const int64_t slots = (int64_t)P.pcg_max_cta_chunks * 9 * 8;
    const int64_t psb = (((int64_t)P.nc * per_cam * w) + 127) & ~(int64_t)127;
    P.pcg_use_ps = (psb + slots <= budget) ? 1 : 0;
    P.pcg_ps_bytes = P.pcg_use_ps ? (int)psb : 0;
    // the staged point pass of the factored form, when the camera rows do not fit
    // in shared memory (their gather from L2 then sits on the direct pass's
    // critical path), with as many stages (2..kMaxStages) as fit.  Where the rows
    // fit, the direct pass is faster (Venice-shaped problem: 109 us per PCG
    // iteration against 134 with two stages, 152 with three stages and the rows
    // in L2, and 147 with a per-warp cp.async prefetch of the next chunk);
    // Final-shaped: 1,318 against 1,475 us with two stages
    const int64_t base = ((P.pcg_ps_bytes + slots) + 127) & ~(int64_t)127;
    const bool ranges_ok = 6 * (int64_t)P.np + 64 < (int64_t)INT32_MAX && (int64_t)P.n + 64 < (int64_t)INT32_MAX;
    int64_t stages = P.fact && !P.pcg_use_ps && P.n_tiles > 0 && ranges_ok ? (budget - base) / kStageBytes : 0;
    if (stages > kMaxStages) stages = kMaxStages;
    if (stages < 2) stages = 0;
    P.pcg_stages = (int)stages;
    P.pcg_stage_off = (int)base;
    P.pcg_smem = stages ? (int)(base + stages * kStageBytes) : (int)(P.pcg_ps_bytes + slots);
}

int pcg_block(const Prob &P) { return P.fp32 ? PcgBlock<float>::value : PcgBlock<double>::value; }

template <bool SR>
static const void *pcg_fn_v(const Prob &P) {
    if (!P.fp32) return (const void *)pcg_kernel<double, true, false, SR>;
    if (P.autodiff) return (const void *)pcg_kernel<float, true, false, SR>;
    return P.pcg_stages ? (const void *)pcg_kernel<float, false, true, SR>
                        : (const void *)pcg_kernel<float, false, false, SR>;
}
static const void *pcg_fn(const Prob &P, int variant = MBA_PCG_STANDARD) {
    return variant == MBA_PCG_SINGLE_REDUCTION ? pcg_fn_v<true>(P) : pcg_fn_v<false>(P);
}

static int resident(const void *fn, int block, size_t smem) {
    int blocks = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, block, smem) != cudaSuccess) return 0;
    return blocks;
}

// One CTA per SM (the camera partition is built for exactly that many);
// returns 0 if either PCG instance (standard, single-reduction) cannot be
// resident with its shared memory.
int pcg_grid_size(const Prob &P) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)P.pcg_smem;
    const bool ok = resident(pcg_fn(P), pcg_block(P), smem) >= 1 &&
                    resident(pcg_fn(P, MBA_PCG_SINGLE_REDUCTION), pcg_block(P), smem) >= 1;
    return ok ? sms : 0;
}

cudaError_t launch_pcg(const Prob &P, int mode, int max_iter, double tol, long long spin_limit, int grid,
                       cudaStream_t s, int forcing, int variant) {
    // the right-hand-side and product-only modes are the standard kernel's
    if (mode != PCG_SOLVE) variant = MBA_PCG_STANDARD;
    const size_t smem = (size_t)P.pcg_smem;
    // the barrier targets count arrivals from zero in every launch
    cudaError_t e = cudaMemsetAsync(&P.st->barrier, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    // the shared-memory plan differs between problems (stages, search direction),
    // so the kernel's dynamic shared-memory limit is set for this launch
    e = cudaFuncSetAttribute(pcg_fn(P, variant), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    Prob Pc = P;
    void *args[] = {(void *)&Pc, (void *)&mode, (void *)&max_iter, (void *)&tol, (void *)&spin_limit, (void *)&forcing};
    return cudaLaunchCooperativeKernel(pcg_fn(P, variant), dim3(grid), dim3(pcg_block(P)), args, smem, s);
}

cudaError_t launch_backsub(const Prob &P, double *partial, int nb, cudaStream_t s) {
    if (P.fact) {
        fact_rows_kernel<<<(P.nc + 127) / 128, 128, 0, s>>>(P, P.x, (float *)P.pT);
        backsub_kernel<float, true><<<nb, kBlock, 0, s>>>(P, partial);
    } else if (P.fp32) {
        backsub_kernel<float, false><<<nb, kBlock, 0, s>>>(P, partial);
    } else {
        backsub_kernel<double, false><<<nb, kBlock, 0, s>>>(P, partial);
    }
    ldec_final_kernel<<<1, kBlock, 0, s>>>(partial, nb, P.st);
    cams_new_kernel<<<(P.nc * 9 + kBlock - 1) / kBlock, kBlock, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace mba
