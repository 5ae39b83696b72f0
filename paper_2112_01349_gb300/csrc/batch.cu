// batch.cu -- batched local bundle adjustment: many independent windows in one
// persistent launch.  Each CTA claims whole windows (largest first, from a
// global counter) and runs, for its window alone, the method of the single
// problem solver:
//   LM loop of Alg. 1 with the trust-region rule of lm.cu,
//   residual / Jacobian / Hessian blocks (Alg. 1; Sec. 3 Eq. 2),
//   Schur elimination (Sec. 3 Eq. 3) and the block-Jacobi PCG of Alg. 2 with
//   the implicit product of Alg. 3, back-substitution (Sec. 3 Eq. 4), FP64
//   cost for accept/reject,
// and, optionally, the adjoint of its solution (as mba_adjoint).  Windows never
// exchange data, so a CTA synchronises only with itself.
//
// Layout.  The camera side of a window (at most 64 cameras: parameters, camera
// tables, B, v, the preconditioner, the PCG vectors, per-warp partial sums)
// lives in shared memory.  Points and observations live in global memory,
// indexed globally; a window's working set is a few hundred KB and stays in L2.
//
// Matrix-free Jacobian.  The point and camera passes recompute the projection
// of each observation from the camera table and the point instead of storing
// J (96 B per observation in FP32): a window is latency- and L2-bound, not
// FP32-bound, so recomputing is the cheaper side of the trade.
//   Jc p  = b_r . (m x X) + D_r . p_t + p_r (d p_f + f r^2 (p_k1 + r^2 p_k2))
//           with m = M p_w per camera, b_r = row r of Jp = D R (of D in the
//           first-order branch), D = d(pixel)/dP;
//   Jc^T s = (M^T (X x g), D^T s, (d, f r^2, f r^4) (p . s)), g = R^T D^T s
//           (D^T s in the first-order branch).
// The IRLS weight W multiplies the products once (W Jp^T Jc p, W Jp b), which
// equals the sqrt(W) scaling of both factors.
//
// Summation orders are fixed by the launch schedule (threads per CTA), so a
// schedule gives the same bits on every run.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>


#include "mba_internal.cuh"

namespace mba {

namespace {

constexpr int kBMaxCams = 64;  // cameras per window
constexpr int kTabS = 29;      // shared-memory stride of a T camera-table row (odd: conflict-free gathers)

struct WinDesc {
    int32_t cam0, nc;    // first camera (global index), count
    int32_t pt0, np;     // first point, count
    int32_t obs0, n;     // first observation of the point- and camera-major regions, count
    int32_t wch0, nwch;  // warp chunks [wch0, wch0 + nwch) and their end entry wch0 + nwch
    int32_t blk0, pad;   // first entry of the window's Schur-block pair offsets (nc (nc + 1) / 2 + 1 entries)
};

struct BatchOpts {
    int32_t max_iter, pcg_max_iter, damping, adjoint, adj_pcg_max, explicit_schur;
    double pcg_tol, initial_radius, min_rel_dec, function_tol, adj_pcg_tol, adj_mu;
    int32_t precond, forcing;  // mba_preconditioner; 1: forcing sequence for the forward solves
    int32_t pcg_variant, pad;  // mba_pcg_variant
};

struct BatchArgs {
    int32_t nw, ncmax, loss, s_smem;  // s_smem: explicit S~ held in shared memory
    double delta;
    const WinDesc *desc;
    const int32_t *order;     // claim order (windows by decreasing observation count)
    int32_t *counter;         // claim counter, zeroed before each launch
    const BatchOpts *opts;
    const int2 *wchunk;       // (first point, first observation) of each warp chunk
    const int2 *pm_pc;        // point-major (point, camera), global indices
    const double2 *pm_uv;     // point-major pixels
    const int32_t *pm_orig;   // point-major -> input index
    const int32_t *cm_pt;     // camera-major point
    const int32_t *cm2pm;     // camera-major -> point-major position
    const int32_t *cam_ptr;   // camera-major offsets per camera (global cameras + 1)
    double *cams, *pts, *pts_new, *dp, *Hll, *wv;
    const int32_t *pm2cm;     // point-major -> camera-major position
    void *Cinv;               // [np][6] T: packed inverse of the damped C~
    void *Wpm;                // [n] T: IRLS weight, point-major (NULL without a loss)
    void *Xw;                 // [np][4] T: the point (per linearisation)
    void *cmX;                // [n][4] T: the observation's point, camera-major (per linearisation)
    void *cms;                // [n] T2: s_k = W Jp b_j, camera-major (per PCG pass)
    // explicit Schur complement (when selected)
    void *Jcm;                // [n][24] T: sqrt(W)-scaled Jc (18) and Jp (6), camera-major (per linearisation)
    const int32_t *blk_ptr;   // pair offsets of each upper 9x9 block (i <= k) of each window
    const int4 *pairs;        // (camera-major position in camera i, in camera k, point, 0), per block
    void *S;                  // per CTA: packed upper blocks of S~ (smax values of T)
    int64_t smax;
    const double *gbar_c, *gbar_p;
    double *grad_obs, *grad_c0, *grad_p0;
    mba_window_summary *out;
    unsigned long long *win_ns;  // per window: nanoseconds its CTA spent on it in the last launch
};

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

// Shared memory of one CTA, carved from the dynamic allocation.
template <typename T>
struct WinMem {
    double *cams, *camn, *tab64, *Hpp, *v, *x, *r, *z, *p, *q, *slot, *sb;
    double *sv;  // s = S~ p of the single-reduction PCG
    T *tabT, *pv, *stage, *BinvT;
    T *rT;  // r rounded to T, the preconditioner's input (FP64: r itself)
    T *S;  // explicit S~ in shared memory (NULL: the CTA's global scratch)
    int32_t *cptr, *wf, *wl, *wcam0;
};

// Pairs staged per warp while a Schur block is formed, and the stride of one
// staged pair (Jc~ of the first observation, F = G Jc~ of the second; padded).
template <typename T>
struct Stage {
    static constexpr int pairs = sizeof(T) == 4 ? 32 : 16;
    static constexpr int stride = 37;
};

template <typename T>
__host__ __device__ inline size_t win_carve(unsigned char *base, int ncmax, int nwarp, int64_t svals, WinMem<T> &m) {
    uintptr_t off = 0;
    const uintptr_t b = (uintptr_t)base;
    auto take = [&](size_t bytes) -> void * {
        void *p = (void *)(b + off);
        off += (bytes + 15) & ~(size_t)15;
        return p;
    };
    const size_t c9 = 9 * (size_t)ncmax;
    m.cams = (double *)take(8 * c9);
    m.camn = (double *)take(8 * c9);
    m.tab64 = (double *)take(8 * (size_t)kCamTab * ncmax);
    m.Hpp = (double *)take(8 * 45 * (size_t)ncmax);
    m.v = (double *)take(8 * c9);
    m.x = (double *)take(8 * c9);
    m.r = (double *)take(8 * c9);
    m.z = (double *)take(8 * c9);
    m.p = (double *)take(8 * c9);
    m.q = (double *)take(8 * c9);
    m.sv = (double *)take(8 * c9);
    // camera-pass slots and the Schur-build staging are never live together
    const size_t slot_b = 8 * 54 * (size_t)(nwarp + ncmax),
                 stage_b = sizeof(T) * Stage<T>::pairs * Stage<T>::stride * (size_t)nwarp;
    m.slot = (double *)take(slot_b > stage_b ? slot_b : stage_b);
    m.stage = (T *)m.slot;
    m.sb = (double *)take(8 * (3 * 32 * (size_t)nwarp + 8));
    m.tabT = (T *)take(sizeof(T) * kTabS * (size_t)ncmax);
    m.pv = (T *)take(sizeof(T) * c9);
    m.rT = sizeof(T) == 8 ? (T *)m.r : (T *)take(sizeof(T) * c9);
    m.cptr = (int32_t *)take(4 * (size_t)(ncmax + 1));
    m.wf = (int32_t *)take(4 * (size_t)ncmax);
    m.wl = (int32_t *)take(4 * (size_t)ncmax);
    m.wcam0 = (int32_t *)take(4 * (size_t)nwarp);
    m.BinvT = (T *)take(sizeof(T) * 45 * (size_t)ncmax);
    m.S = svals > 0 ? (T *)take(sizeof(T) * (size_t)svals) : nullptr;
    return (size_t)off;
}

// Per-window control state (shared, written by thread 0 between barriers).
struct WinState {
    double radius, factor, mu, F, F0, Fn, ldec, mu_acc;
    double g0;  // norm of the window's first reduced right-hand side (forcing sequence)
    int32_t win, relin, done, iter, acc_total, pcg_total, status, accept, adj_iters;
    int32_t blockfail;  // a damped block was not positive definite (this iteration)
};

__device__ __forceinline__ double damp_term_b(int damping, double d) {
    if (damping == MBA_DAMP_IDENTITY) return 1.0;
    return fmin(fmax(d, 1e-6), 1e32);
}

// Block-wide sums of two doubles; every thread gets the result.  Fixed order:
// the per-thread values go through shared memory, warp 0 adds them (lane l
// takes threads l, l + 32, ...) and finishes with a butterfly.  One warp does
// all the FP64 additions: on this GPU each warp-wide FP64 instruction holds
// the SM's FP64 pipe for 16 cycles, so spreading the tree over every warp costs
// several times more pipe time.  sb holds 2 NT + 2 doubles.
template <int NT>
__device__ __forceinline__ double2 cta_sum2(double a, double b, double *sb) {
    sb[threadIdx.x] = a;
    sb[NT + threadIdx.x] = b;
    __syncthreads();
    if (threadIdx.x < 32) {
        // pairwise tree over the NT / 32 values of the lane (short dependency chain)
        const int lane = threadIdx.x;
        double xv[NT / 32], yv[NT / 32];
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) {
            xv[k] = sb[lane + 32 * k];
            yv[k] = sb[NT + lane + 32 * k];
        }
#pragma unroll
        for (int h = NT / 64; h > 0; h >>= 1)
#pragma unroll
            for (int k = 0; k < h; ++k) {
                xv[k] += xv[k + h];
                yv[k] += yv[k + h];
            }
        double x = xv[0], y = yv[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (lane == 0) {
            sb[2 * NT] = x;
            sb[2 * NT + 1] = y;
        }
    }
    __syncthreads();
    return make_double2(sb[2 * NT], sb[2 * NT + 1]);
}

// The same sum, with fin(x, y) run by thread 0 on the result before the
// closing barrier (the PCG's scalar recurrences: one thread evaluates the
// divisions and square roots and publishes the outcome in shared memory).
template <int NT, typename F>
__device__ __forceinline__ void cta_sum2f(double a, double b, double *sb, F &&fin) {
    sb[threadIdx.x] = a;
    sb[NT + threadIdx.x] = b;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double xv[NT / 32], yv[NT / 32];
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) {
            xv[k] = sb[lane + 32 * k];
            yv[k] = sb[NT + lane + 32 * k];
        }
#pragma unroll
        for (int h = NT / 64; h > 0; h >>= 1)
#pragma unroll
            for (int k = 0; k < h; ++k) {
                xv[k] += xv[k + h];
                yv[k] += yv[k + h];
            }
        double x = xv[0], y = yv[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (lane == 0) fin(x, y);
    }
    __syncthreads();
}

// Three sums with fin(x, y, z) run by thread 0 before the closing barrier
// (the single-reduction PCG takes r.r, r.u and w.u in one pass).  sb holds
// 3 NT values; the same fixed order as cta_sum2f.
template <int NT, typename F>
__device__ __forceinline__ void cta_sum3f(double a, double b, double c, double *sb, F &&fin) {
    sb[threadIdx.x] = a;
    sb[NT + threadIdx.x] = b;
    sb[2 * NT + threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double xv[NT / 32], yv[NT / 32], zv[NT / 32];
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) {
            xv[k] = sb[lane + 32 * k];
            yv[k] = sb[NT + lane + 32 * k];
            zv[k] = sb[2 * NT + lane + 32 * k];
        }
#pragma unroll
        for (int h = NT / 64; h > 0; h >>= 1)
#pragma unroll
            for (int k = 0; k < h; ++k) {
                xv[k] += xv[k + h];
                yv[k] += yv[k + h];
                zv[k] += zv[k + h];
            }
        double x = xv[0], y = yv[0], z = zv[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
            z += __shfl_xor_sync(0xffffffffu, z, o);
        }
        if (lane == 0) fin(x, y, z);
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void ld_c(const T *Ci, int pt, T *c) {
    using T2 = typename V2<T>::type;
    const T2 *p = reinterpret_cast<const T2 *>(Ci + 6 * (int64_t)pt);
    const T2 a = p[0], b = p[1], e = p[2];
    c[0] = a.x;
    c[1] = a.y;
    c[2] = b.x;
    c[3] = b.y;
    c[4] = e.x;
    c[5] = e.y;
}

template <typename T>
__device__ __forceinline__ void sym3_mul(const T *c, T a0, T a1, T a2, T *b) {
    b[0] = c[0] * a0 + c[1] * a1 + c[2] * a2;
    b[1] = c[1] * a0 + c[3] * a1 + c[4] * a2;
    b[2] = c[2] * a0 + c[4] * a1 + c[5] * a2;
}

// Projection of one observation with the pieces of its Jacobian that the
// matrix-free passes need: the normalised point p, r^2, the distortion d,
// D = d(pixel)/dP (2x3) and Jp = D R; e = pi - u if RES.  Same arithmetic as
// project<T, true> for e, D and Jp.
template <typename T>
struct ObsJ {
    T px, py, r2, d;
    T D[6], Jp[6];
    T e0, e1;
};

template <typename T, bool RES>
__device__ __forceinline__ void obs_jac(const T *ct, T X0, T X1, T X2, T u0, T u1, ObsJ<T> &o) {
    const T R0 = ct[0], R1 = ct[1], R2 = ct[2], R3 = ct[3], R4 = ct[4], R5 = ct[5], R6 = ct[6], R7 = ct[7],
            R8 = ct[8];
    const T P0 = R0 * X0 + R1 * X1 + R2 * X2 + ct[18];
    const T P1 = R3 * X0 + R4 * X1 + R5 * X2 + ct[19];
    const T P2 = R6 * X0 + R7 * X1 + R8 * X2 + ct[20];
    const T iz = rcp_rn(P2);
    const T px = -P0 * iz, py = -P1 * iz;
    const T f = ct[21], k1 = ct[22], k2 = ct[23];
    const T r2 = px * px + py * py;
    const T d = T(1) + k1 * r2 + k2 * r2 * r2;
    if (RES) {
        o.e0 = f * d * px - u0;
        o.e1 = f * d * py - u1;
    }
    const T dd = T(2) * k1 + T(4) * k2 * r2;
    const T a00 = f * (d + dd * px * px), a01 = f * dd * px * py, a11 = f * (d + dd * py * py);
    o.D[0] = -a00 * iz;
    o.D[1] = -a01 * iz;
    o.D[2] = -(a00 * px + a01 * py) * iz;
    o.D[3] = -a01 * iz;
    o.D[4] = -a11 * iz;
    o.D[5] = -(a01 * px + a11 * py) * iz;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        o.Jp[r * 3 + 0] = o.D[r * 3] * R0 + o.D[r * 3 + 1] * R3 + o.D[r * 3 + 2] * R6;
        o.Jp[r * 3 + 1] = o.D[r * 3] * R1 + o.D[r * 3 + 1] * R4 + o.D[r * 3 + 2] * R7;
        o.Jp[r * 3 + 2] = o.D[r * 3] * R2 + o.D[r * 3 + 1] * R5 + o.D[r * 3 + 2] * R8;
    }
    o.px = px;
    o.py = py;
    o.r2 = r2;
    o.d = d;
}

// t = Jc v for the camera vector v given as pv = (M v_w, v_t, v_f, v_k1, v_k2).
template <typename T>
__device__ __forceinline__ void jc_apply(const T *ct, const T *pv, const ObsJ<T> &o, T X0, T X1, T X2, T &t0,
                                         T &t1) {
    const T c0 = pv[1] * X2 - pv[2] * X1, c1 = pv[2] * X0 - pv[0] * X2, c2 = pv[0] * X1 - pv[1] * X0;
    const bool small = ct[24] != T(0);
    const T *b = small ? o.D : o.Jp;
    const T kap = o.d * pv[6] + ct[21] * o.r2 * (pv[7] + o.r2 * pv[8]);
    t0 = b[0] * c0 + b[1] * c1 + b[2] * c2 + o.D[0] * pv[3] + o.D[1] * pv[4] + o.D[2] * pv[5] + o.px * kap;
    t1 = b[3] * c0 + b[4] * c1 + b[5] * c2 + o.D[3] * pv[3] + o.D[4] * pv[4] + o.D[5] * pv[5] + o.py * kap;
}

// y = Jc^T s by the transposed chain rule (no Jc formed).
template <typename T>
__device__ __forceinline__ void jct_apply(const T *ct, T X0, T X1, T X2, T s0, T s1, T *y) {
    const T P0 = ct[0] * X0 + ct[1] * X1 + ct[2] * X2 + ct[18];
    const T P1 = ct[3] * X0 + ct[4] * X1 + ct[5] * X2 + ct[19];
    const T P2 = ct[6] * X0 + ct[7] * X1 + ct[8] * X2 + ct[20];
    const T iz = rcp_rn(P2);
    const T px = -P0 * iz, py = -P1 * iz;
    const T f = ct[21], k1 = ct[22], k2 = ct[23];
    const T r2 = px * px + py * py;
    const T d = T(1) + k1 * r2 + k2 * r2 * r2;
    const T dd = T(2) * k1 + T(4) * k2 * r2;
    const T a00 = f * (d + dd * px * px), a01 = f * dd * px * py, a11 = f * (d + dd * py * py);
    const T g0 = -(a00 * s0 + a01 * s1) * iz, g1 = -(a01 * s0 + a11 * s1) * iz;
    const T v0 = g0, v1 = g1, v2 = g0 * px + g1 * py;  // D^T s
    y[3] = v0;
    y[4] = v1;
    y[5] = v2;
    T w0 = v0, w1 = v1, w2 = v2;
    if (ct[24] == T(0)) {
        w0 = ct[0] * v0 + ct[3] * v1 + ct[6] * v2;
        w1 = ct[1] * v0 + ct[4] * v1 + ct[7] * v2;
        w2 = ct[2] * v0 + ct[5] * v1 + ct[8] * v2;
    }
    const T u0 = X1 * w2 - X2 * w1, u1 = X2 * w0 - X0 * w2, u2 = X0 * w1 - X1 * w0;
    y[0] = ct[9] * u0 + ct[12] * u1 + ct[15] * u2;
    y[1] = ct[10] * u0 + ct[13] * u1 + ct[16] * u2;
    y[2] = ct[11] * u0 + ct[14] * u1 + ct[17] * u2;
    const T pss = px * s0 + py * s1;
    y[6] = d * pss;
    y[7] = f * r2 * pss;
    y[8] = f * r2 * r2 * pss;
}

// Inclusive segmented scan over the lanes of a warp; segments are runs of
// equal keys (whole points, contiguous).
template <typename T, int K>
__device__ __forceinline__ void seg_scan(T *u, int key, int lane) {
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const int kp = __shfl_up_sync(0xffffffffu, key, dd);
        T v[K];
#pragma unroll
        for (int q = 0; q < K; ++q) v[q] = __shfl_up_sync(0xffffffffu, u[q], dd);
        if (lane >= dd && kp == key)
#pragma unroll
            for (int q = 0; q < K; ++q) u[q] += v[q];
    }
}

template <typename T, int K>
__device__ __forceinline__ void warp_allsum(T *u) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < K; ++q) u[q] += __shfl_xor_sync(0xffffffffu, u[q], o);
}

// Per-observation records, rewritten once per linearisation (X) or per damped
// solve (C~^-1, W, key) so that the PCG passes read them coalesced, one level
// of indirection deep, instead of gathering per point.
template <typename T>
__device__ __forceinline__ void ld4(const T *p, T &a, T &b, T &c, T &d);
template <>
__device__ __forceinline__ void ld4<float>(const float *p, float &a, float &b, float &c, float &d) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = v.x;
    b = v.y;
    c = v.z;
    d = v.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double *p, double &a, double &b, double &c, double &d) {
    const double2 u = reinterpret_cast<const double2 *>(p)[0], v = reinterpret_cast<const double2 *>(p)[1];
    a = u.x;
    b = u.y;
    c = v.x;
    d = v.y;
}
template <typename T>
__device__ __forceinline__ void st4(T *p, T a, T b, T c, T d);
template <>
__device__ __forceinline__ void st4<float>(float *p, float a, float b, float c, float d) {
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void st4<double>(double *p, double a, double b, double c, double d) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
}
template <typename T>
struct PmRec {
    T X0, X1, X2, W;
    T c[6];
    int key;  // (local point << 6) | local camera
    int cm;   // camera-major position of the observation
};

// Per-observation words of a record (coalesced): (point, camera), the
// camera-major position and the IRLS weight.
template <typename T>
__device__ __forceinline__ void load_idx(const BatchArgs &A, int o, int2 &pc, int &cm, T &W) {
    pc = __ldg(A.pm_pc + o);
    cm = __ldg(A.pm2cm + o);
    W = A.Wpm ? ((const T *)A.Wpm)[o] : T(1);
}

// Per-point words of a record (gathered; lanes of one point share them):
// the point in T and the packed C~^-1.
template <typename T>
__device__ __forceinline__ void load_pt(const BatchArgs &A, const WinDesc &d, int2 pc, int cm, T W, PmRec<T> &r) {
    T unused;
    ld4<T>((const T *)A.Xw + 4 * (int64_t)pc.x, r.X0, r.X1, r.X2, unused);
    ld_c<T>((const T *)A.Cinv, pc.x, r.c);
    r.W = W;
    r.cm = cm;
    r.key = ((pc.x - d.pt0) << 6) | (pc.y - d.cam0);
}

template <typename T>
__device__ __forceinline__ void load_rec(const BatchArgs &A, const WinDesc &d, int o, PmRec<T> &r) {
    int2 pc;
    int cm;
    T W;
    load_idx<T>(A, o, pc, cm, W);
    load_pt<T>(A, d, pc, cm, W, r);
}

// Linearisation over the window's warp chunks: e, Jp and W per observation; per point
// C = sum W Jp^T Jp and w = -sum W Jp^T e by a segmented scan (whole points per
// chunk) or a warp sum (one long-track point); the point-major X record and W.
template <typename T, int NT>
__device__ void lin_points(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    T *Xw = (T *)A.Xw;
    T *Wpm = (T *)A.Wpm;
    const T delta = (T)A.delta;
    for (int c = d.wch0 + wid; c < d.wch0 + d.nwch; c += NW) {
        const int2 c0 = __ldg(A.wchunk + c), c1 = __ldg(A.wchunk + c + 1);
        const int o0 = c0.y, m = c1.y - c0.y;
        const bool longp = m > 32;
        T h[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) h[q] = T(0);
        int key = -1 - lane, pt = c0.x;
        for (int base = 0; base < m; base += 32) {
            const bool act = base + lane < m;
            const int o = o0 + base + (act ? lane : 0);
            const int2 pc = __ldg(A.pm_pc + o);
            pt = pc.x;
            if (act) key = pc.x;
            const T X0 = (T)A.pts[3 * (int64_t)pt], X1 = (T)A.pts[3 * (int64_t)pt + 1],
                    X2 = (T)A.pts[3 * (int64_t)pt + 2];
            const double2 uv = __ldg(A.pm_uv + o);
            T e[2], Jc[18], Jp[6];
            project<T, true>(M.tabT + (pc.y - d.cam0) * kTabS, X0, X1, X2, (T)uv.x, (T)uv.y, e, Jc, Jp);
            T rho, W;
            loss_weight<T>(A.loss, delta, e[0] * e[0] + e[1] * e[1], &rho, &W);
            if (act) {
                T jw[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) jw[q] = W * Jp[q];
                h[0] += jw[0] * Jp[0] + jw[3] * Jp[3];
                h[1] += jw[0] * Jp[1] + jw[3] * Jp[4];
                h[2] += jw[0] * Jp[2] + jw[3] * Jp[5];
                h[3] += jw[1] * Jp[1] + jw[4] * Jp[4];
                h[4] += jw[1] * Jp[2] + jw[4] * Jp[5];
                h[5] += jw[2] * Jp[2] + jw[5] * Jp[5];
                h[6] -= jw[0] * e[0] + jw[3] * e[1];
                h[7] -= jw[1] * e[0] + jw[4] * e[1];
                h[8] -= jw[2] * e[0] + jw[5] * e[1];
                if (Wpm) Wpm[o] = W;
            }
        }
        bool tail;
        if (longp) {
            warp_allsum<T, 9>(h);
            tail = lane == 0;
            pt = c0.x;
        } else {
            seg_scan<T, 9>(h, key, lane);
            const int nxt = __shfl_down_sync(full, key, 1);
            tail = lane < m && (lane == 31 || lane == m - 1 || nxt != key);
        }
        if (tail) {
#pragma unroll
            for (int q = 0; q < 6; ++q) A.Hll[6 * (int64_t)pt + q] = (double)h[q];
#pragma unroll
            for (int q = 0; q < 3; ++q) A.wv[3 * (int64_t)pt + q] = (double)h[6 + q];
            st4<T>(Xw + 4 * (int64_t)pt, (T)A.pts[3 * (int64_t)pt], (T)A.pts[3 * (int64_t)pt + 1],
                   (T)A.pts[3 * (int64_t)pt + 2], T(0));
        }
    }
}

// Right-hand side pass, per observation (no segments): s_k = W Jp b_j with
// b_j = C~_j^-1 wvec_j, into camera-major order.
template <typename T, int NT>
__device__ void rhs_points(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d, const double *wvec) {
    using T2 = typename V2<T>::type;
    T2 *cms = (T2 *)A.cms;
    for (int k = threadIdx.x; k < d.n; k += NT) {
        PmRec<T> r;
        load_rec<T>(A, d, d.obs0 + k, r);
        const int pt = d.pt0 + (r.key >> 6);
        ObsJ<T> J;
        obs_jac<T, false>(M.tabT + (r.key & 63) * kTabS, r.X0, r.X1, r.X2, T(0), T(0), J);
        T b[3];
        sym3_mul<T>(r.c, (T)wvec[3 * (int64_t)pt], (T)wvec[3 * (int64_t)pt + 1], (T)wvec[3 * (int64_t)pt + 2], b);
        T2 sv;
        sv.x = r.W * (J.Jp[0] * b[0] + J.Jp[1] * b[1] + J.Jp[2] * b[2]);
        sv.y = r.W * (J.Jp[3] * b[0] + J.Jp[4] * b[1] + J.Jp[5] * b[2]);
        cms[r.cm] = sv;
    }
}

// u_k = W Jp^T (Jc v) for one record (v given by its pv row)
template <typename T>
__device__ __forceinline__ void rec_u(const WinMem<T> &M, const PmRec<T> &r, ObsJ<T> &J, T &a0, T &a1, T *u) {
    const int lc = r.key & 63;
    const T *ct = M.tabT + lc * kTabS;
    obs_jac<T, false>(ct, r.X0, r.X1, r.X2, T(0), T(0), J);
    jc_apply<T>(ct, M.pv + lc * 9, J, r.X0, r.X1, r.X2, a0, a1);
    const T tw0 = r.W * a0, tw1 = r.W * a1;
    u[0] = J.Jp[0] * tw0 + J.Jp[3] * tw1;
    u[1] = J.Jp[1] * tw0 + J.Jp[4] * tw1;
    u[2] = J.Jp[2] * tw0 + J.Jp[5] * tw1;
}

// The E^T p, C~^-1, E pass of Alg. 3: s_k = W Jp b_j, b_j = C~_j^-1 sum_k u_k,
// stored camera-major.  The records of the next chunk are loaded before the
// current chunk is computed (software pipelining over the warp's chunks).
template <typename T, int NT>
__device__ void iter_points(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d) {
    using T2 = typename V2<T>::type;
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    T2 *cms = (T2 *)A.cms;
    const int cend = d.wch0 + d.nwch;
    int c = d.wch0 + wid;
    if (c >= cend) return;
    // three-deep pipeline over the warp's chunks: chunk c computed, chunk c+NW's
    // per-point gathers and chunk c+2NW's per-observation words in flight,
    // chunk c+3NW's bounds read
    auto lane_obs = [&](int2 a0, int2 a1) { return a0.y + ((lane < a1.y - a0.y) ? lane : 0); };
    int2 mc = __ldg(A.wchunk + c), mc1 = __ldg(A.wchunk + c + 1);
    PmRec<T> cur;
    load_rec<T>(A, d, lane_obs(mc, mc1), cur);
    bool hn = c + NW < cend, hm = c + 2 * NW < cend;
    int2 mn = mc1, mn1 = mc1, mm = mc1, mm1 = mc1, pcn = make_int2(0, 0);
    int cmn = 0;
    T Wn = T(1);
    if (hn) {
        mn = __ldg(A.wchunk + c + NW);
        mn1 = __ldg(A.wchunk + c + NW + 1);
        load_idx<T>(A, lane_obs(mn, mn1), pcn, cmn, Wn);
    }
    if (hm) {
        mm = __ldg(A.wchunk + c + 2 * NW);
        mm1 = __ldg(A.wchunk + c + 2 * NW + 1);
    }
    for (;;) {
        PmRec<T> nxt;
        if (hn) load_pt<T>(A, d, pcn, cmn, Wn, nxt);
        int2 pcm = make_int2(0, 0);
        int cmm = 0;
        T Wm = T(1);
        if (hm) load_idx<T>(A, lane_obs(mm, mm1), pcm, cmm, Wm);
        const bool hq = c + 3 * NW < cend;
        int2 mq = mm1, mq1 = mm1;
        if (hq) {
            mq = __ldg(A.wchunk + c + 3 * NW);
            mq1 = __ldg(A.wchunk + c + 3 * NW + 1);
        }
        const int o0 = mc.y, m = mc1.y - mc.y;
        if (m <= 32) {
            const bool act = lane < m;
            const int key = act ? (cur.key >> 6) : -1 - lane;
            ObsJ<T> J;
            T a0, a1, u[3];
            rec_u<T>(M, cur, J, a0, a1, u);
            seg_scan<T, 3>(u, key, lane);
            const int kn = __shfl_down_sync(full, key, 1);
            const bool tail = act && (lane == 31 || lane == m - 1 || kn != key);
            const unsigned tails = __ballot_sync(full, tail);
            const unsigned mine = tails & (0xffffffffu << lane);
            const int src = mine ? __ffs(mine) - 1 : lane;
            T bt[3], b[3];
            sym3_mul<T>(cur.c, u[0], u[1], u[2], bt);
#pragma unroll
            for (int q = 0; q < 3; ++q) b[q] = __shfl_sync(full, bt[q], src);
            if (act) {
                T2 sv;
                sv.x = cur.W * (J.Jp[0] * b[0] + J.Jp[1] * b[1] + J.Jp[2] * b[2]);
                sv.y = cur.W * (J.Jp[3] * b[0] + J.Jp[4] * b[1] + J.Jp[5] * b[2]);
                cms[cur.cm] = sv;
            }
        } else {
            // one point with a long track: two sweeps over 32-observation slices
            T a[3] = {T(0), T(0), T(0)};
            T cc[6];
            for (int base = 0; base < m; base += 32) {
                if (base + lane < m) {
                    PmRec<T> r;
                    load_rec<T>(A, d, o0 + base + lane, r);
                    ObsJ<T> J;
                    T a0, a1, u[3];
                    rec_u<T>(M, r, J, a0, a1, u);
                    a[0] += u[0];
                    a[1] += u[1];
                    a[2] += u[2];
                }
            }
            warp_allsum<T, 3>(a);
            PmRec<T> r0;
            load_rec<T>(A, d, o0, r0);
#pragma unroll
            for (int q = 0; q < 6; ++q) cc[q] = r0.c[q];
            T b[3];
            sym3_mul<T>(cc, a[0], a[1], a[2], b);
            for (int base = 0; base < m; base += 32) {
                if (base + lane < m) {
                    PmRec<T> r;
                    load_rec<T>(A, d, o0 + base + lane, r);
                    ObsJ<T> J;
                    obs_jac<T, false>(M.tabT + (r.key & 63) * kTabS, r.X0, r.X1, r.X2, T(0), T(0), J);
                    T2 sv;
                    sv.x = r.W * (J.Jp[0] * b[0] + J.Jp[1] * b[1] + J.Jp[2] * b[2]);
                    sv.y = r.W * (J.Jp[3] * b[0] + J.Jp[4] * b[1] + J.Jp[5] * b[2]);
                    cms[r.cm] = sv;
                }
            }
        }
        if (!hn) break;
        c += NW;
        cur = nxt;
        mc = mn;
        mc1 = mn1;
        mn = mm;
        mn1 = mm1;
        pcn = pcm;
        cmn = cmm;
        Wn = Wm;
        hn = hm;
        mm = mq;
        mm1 = mq1;
        hm = hq;
    }
}

// Back-substitution (Sec. 3 Eq. 4): dp_j = C~_j^-1 (wvec_j - sum_k W Jp^T Jc x),
// d_k = Jc x + Jp dp_j.  Forward solve: candidate points and this thread's
// share of the model decrease sum_k W (-e.d - |d|^2/2).  Adjoint: W d_k per
// observation in input order.
template <typename T, int NT>
__device__ double back_points(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d, const double *wvec,
                              bool adj) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    double ldec = 0.0;
    for (int c = d.wch0 + wid; c < d.wch0 + d.nwch; c += NW) {
        const int2 c0 = __ldg(A.wchunk + c), c1 = __ldg(A.wchunk + c + 1);
        const int o0 = c0.y, m = c1.y - c0.y;
        // first sweep: u sums (segmented for whole-point chunks, warp-wide for a long track)
        T u[3] = {T(0), T(0), T(0)};
        int key = -1 - lane;
        PmRec<T> r;
        T a0 = T(0), a1 = T(0);
        ObsJ<T> J;
        for (int base = 0; base < m; base += 32) {
            const bool act = base + lane < m;
            load_rec<T>(A, d, o0 + base + (act ? lane : 0), r);
            T uu[3];
            rec_u<T>(M, r, J, a0, a1, uu);
            if (act) {
                key = r.key >> 6;
                u[0] += uu[0];
                u[1] += uu[1];
                u[2] += uu[2];
            }
        }
        T b[3];
        bool tail;
        int ptl;
        if (m > 32) {
            warp_allsum<T, 3>(u);
            tail = lane == 0;
            ptl = c0.x - d.pt0;
        } else {
            seg_scan<T, 3>(u, key, lane);
            const int kn = __shfl_down_sync(full, key, 1);
            tail = lane < m && (lane == 31 || lane == m - 1 || kn != key);
            ptl = key;
        }
        const unsigned tails = __ballot_sync(full, tail);
        const unsigned mine = tails & (0xffffffffu << lane);
        const int src = m > 32 ? 0 : (mine ? __ffs(mine) - 1 : lane);
        {
            T bt[3];
            const int64_t pt = (int64_t)d.pt0 + (ptl >= 0 ? ptl : 0);
            sym3_mul<T>(r.c, (T)wvec[3 * pt] - u[0], (T)wvec[3 * pt + 1] - u[1], (T)wvec[3 * pt + 2] - u[2], bt);
            if (tail) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    A.dp[3 * pt + q] = (double)bt[q];
                    if (!adj) A.pts_new[3 * pt + q] = A.pts[3 * pt + q] + (double)bt[q];
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) b[q] = __shfl_sync(full, bt[q], src);
        }
        // second sweep: d_k (the records of a whole-point chunk are still in registers)
        for (int base = 0; base < m; base += 32) {
            const bool act = base + lane < m;
            const int o = o0 + base + (act ? lane : 0);
            if (m > 32) {
                load_rec<T>(A, d, o, r);
                T uu[3];
                rec_u<T>(M, r, J, a0, a1, uu);
            }
            if (act) {
                const T dd0 = a0 + J.Jp[0] * b[0] + J.Jp[1] * b[1] + J.Jp[2] * b[2];
                const T dd1 = a1 + J.Jp[3] * b[0] + J.Jp[4] * b[1] + J.Jp[5] * b[2];
                if (adj) {
                    const int64_t k = __ldg(A.pm_orig + o);
                    A.grad_obs[2 * k] = (double)r.W * (double)dd0;
                    A.grad_obs[2 * k + 1] = (double)r.W * (double)dd1;
                } else {
                    const double2 uv = __ldg(A.pm_uv + o);
                    ObsJ<T> Je;
                    obs_jac<T, true>(M.tabT + (r.key & 63) * kTabS, r.X0, r.X1, r.X2, (T)uv.x, (T)uv.y, Je);
                    const double e0 = (double)Je.e0, e1 = (double)Je.e1, x0 = (double)dd0, x1 = (double)dd1;
                    ldec += (double)r.W * (-(e0 * x0 + e1 * x1) - 0.5 * (x0 * x0 + x1 * x1));
                }
            }
        }
    }
    return ldec;
}

// Camera-major pass: warp w owns observations [lo(w), lo(w+1)) of the window
// (lo(w) = w n / NW), split at camera boundaries into segments; each segment's
// sum goes to slot (w + camera), a slot no other segment uses.  LIN: the 45
// entries of B = sum W Jc^T Jc and v = -sum W Jc^T e (54 per slot);
// otherwise sum Jc^T s (9 per slot).
template <typename T, int NT, bool LIN>
__device__ void camera_pass(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d, bool wj = false) {
    using T2 = typename V2<T>::type;
    constexpr int NW = NT / 32;
    constexpr int K = LIN ? 54 : 9;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int lo = (int)(((int64_t)wid * d.n) / NW), hi = (int)(((int64_t)(wid + 1) * d.n) / NW);
    if (lo >= hi) return;
    T *cmX = (T *)A.cmX;
    const T2 *cms = (const T2 *)A.cms;
    const T delta = (T)A.delta;
    int cam = M.wcam0[wid];
    int beg = lo;
    for (;;) {
        const int end = min(hi, M.cptr[cam + 1]);
        const T *ct = M.tabT + cam * kTabS;
        T acc[K];
#pragma unroll
        for (int q = 0; q < K; ++q) acc[q] = T(0);
        if (LIN) {
            for (int c = beg + lane; c < end; c += 32) {
                const int gc = d.obs0 + c;
                const int pt = __ldg(A.cm_pt + gc), pm = __ldg(A.cm2pm + gc);
                const T X0 = (T)A.pts[3 * (int64_t)pt], X1 = (T)A.pts[3 * (int64_t)pt + 1],
                        X2 = (T)A.pts[3 * (int64_t)pt + 2];
                st4<T>(cmX + 4 * (int64_t)gc, X0, X1, X2, T(0));
                const double2 uv = __ldg(A.pm_uv + pm);
                T e[2], Jc[18], Jp[6];
                project<T, true>(ct, X0, X1, X2, (T)uv.x, (T)uv.y, e, Jc, Jp);
                T rho, W;
                loss_weight<T>(A.loss, delta, e[0] * e[0] + e[1] * e[1], &rho, &W);
                if (wj) {
                    const T sw = sqrt(W);
                    T *jo = (T *)A.Jcm + 24 * (int64_t)gc;
#pragma unroll
                    for (int q = 0; q < 16; q += 4) st4<T>(jo + q, sw * Jc[q], sw * Jc[q + 1], sw * Jc[q + 2], sw * Jc[q + 3]);
                    st4<T>(jo + 16, sw * Jc[16], sw * Jc[17], sw * Jp[0], sw * Jp[1]);
                    st4<T>(jo + 20, sw * Jp[2], sw * Jp[3], sw * Jp[4], sw * Jp[5]);
                }
                int idx = 0;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const T w0 = W * Jc[a], w1 = W * Jc[9 + a];
#pragma unroll
                    for (int b = a; b < 9; ++b) acc[idx++] += w0 * Jc[b] + w1 * Jc[9 + b];
                    acc[45 + a] -= w0 * e[0] + w1 * e[1];
                }
            }
        } else {
            // the next step's X and s are loaded before the current step is computed
            int c = beg + lane;
            T X0 = T(0), X1 = T(0), X2 = T(0), unused;
            T2 sv;
            sv.x = T(0);
            sv.y = T(0);
            if (c < end) {
                ld4<T>(cmX + 4 * (int64_t)(d.obs0 + c), X0, X1, X2, unused);
                sv = cms[d.obs0 + c];
            }
            for (; c < end; c += 32) {
                const T x0 = X0, x1 = X1, x2 = X2;
                const T2 s_ = sv;
                if (c + 32 < end) {
                    ld4<T>(cmX + 4 * (int64_t)(d.obs0 + c + 32), X0, X1, X2, unused);
                    sv = cms[d.obs0 + c + 32];
                }
                T y[9];
                jct_apply<T>(ct, x0, x1, x2, s_.x, s_.y, y);
#pragma unroll
                for (int q = 0; q < K; ++q) acc[q] += y[q];
            }
        }
        warp_allsum<T, K>(acc);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < K; ++q) M.slot[(wid + cam) * K + q] = (double)acc[q];
        if (end >= hi) break;
        beg = end;
        ++cam;
    }
}

// Sum of camera i's segment slots (stride K), in warp order.
__device__ __forceinline__ double slot_sum(const double *slot, const int32_t *wf, const int32_t *wl, int i, int K,
                                           int q) {
    double s = 0.0;
    for (int w = wf[i]; w <= wl[i]; ++w) s += slot[(w + i) * K + q];
    return s;
}

// (M v_w, v_t, v_f, v_k1, v_k2) per camera in T, for jc_apply.
template <typename T, int NT>
__device__ __forceinline__ void make_pv(const WinMem<T> &M, const double *vec, int nc) {
    for (int t = threadIdx.x; t < 9 * nc; t += NT) {
        const int i = t / 9, a = t - 9 * (t / 9);
        T val;
        if (a < 3) {
            const T *Mr = M.tabT + i * kTabS + 9 + 3 * a;
            val = Mr[0] * (T)vec[9 * i] + Mr[1] * (T)vec[9 * i + 1] + Mr[2] * (T)vec[9 * i + 2];
        } else {
            val = (T)vec[t];
        }
        M.pv[t] = val;
    }
}

// z = B~^-1 r per camera, with B~^-1 (inverted in FP64) applied in the
// problem's precision T to M.rT, the T copy of r that every update of r keeps
// (one conversion per entry instead of nine); returns (r.r, r.z) partials in
// FP64.
template <typename T, int NT>
__device__ __forceinline__ double2 precond(const WinMem<T> &M, int nc) {
    double rr = 0.0, rz = 0.0;
    for (int t = threadIdx.x; t < 9 * nc; t += NT) {
        const int i = t / 9, a = t - 9 * (t / 9);
        const T *Bi = M.BinvT + 45 * i;
        const T *ri = M.rT + 9 * i;
        T zt = T(0);
#pragma unroll
        for (int b = 0; b < 9; ++b) zt = fma(Bi[sym9(a, b)], ri[b], zt);
        const double z = (double)zt;
        M.z[t] = z;
        rr = fma(M.r[t], M.r[t], rr);
        rz = fma(M.r[t], z, rz);
    }
    return make_double2(rr, rz);
}

template <typename T, int NT>
__device__ void linearize(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d, bool xs) {
    for (int t = threadIdx.x; t < d.nc * kCamTab; t += NT) {
        const int i = t / kCamTab, q = t - kCamTab * (t / kCamTab);
        M.tabT[i * kTabS + q] = (T)M.tab64[t];
    }
    __syncthreads();
    lin_points<T, NT>(A, M, d);
    __syncthreads();
    camera_pass<T, NT, true>(A, M, d, xs);
    __syncthreads();
    for (int t = threadIdx.x; t < d.nc * 54; t += NT) {
        const int i = t / 54, q = t - 54 * (t / 54);
        const double s = slot_sum(M.slot, M.wf, M.wl, i, 54, q);
        if (q < 45) M.Hpp[45 * i + q] = s;
        else M.v[9 * i + (q - 45)] = s;
    }
    __syncthreads();
}

// B~ = B + mu D and its inverse (Cholesky, FP64, packed), C~^-1 per point (adjugate, FP64 -> T).
template <typename T, int NT>
__device__ void damp(const BatchArgs &A, const WinMem<T> &M, WinState &S, const WinDesc &d, double mu, int damping) {
    for (int i = threadIdx.x; i < d.nc; i += NT) {
        double L[81];
        for (int a = 0; a < 9; ++a)
            for (int b = 0; b < 9; ++b) L[a * 9 + b] = M.Hpp[45 * i + sym9(a, b)];
        for (int a = 0; a < 9; ++a) L[a * 10] += mu * damp_term_b(damping, L[a * 10]);
        bool ok = true;
        double il[9];  // reciprocals of the Cholesky diagonal
        for (int j = 0; j < 9 && ok; ++j) {
            double s = L[j * 9 + j];
            for (int k = 0; k < j; ++k) s -= L[j * 9 + k] * L[j * 9 + k];
            if (!(s > 0.0) || !isfinite(s)) {
                ok = false;
                break;
            }
            const double l = sqrt(s);
            il[j] = 1.0 / l;
            L[j * 9 + j] = l;
            for (int r = j + 1; r < 9; ++r) {
                double t = L[r * 9 + j];
                for (int k = 0; k < j; ++k) t -= L[r * 9 + k] * L[j * 9 + k];
                L[r * 9 + j] = t * il[j];
            }
        }
        if (!ok) {
            S.blockfail = 1;
            continue;
        }
        for (int col = 0; col < 9; ++col) {
            double y[9];
            for (int r = 0; r < 9; ++r) {
                double s = (r == col) ? 1.0 : 0.0;
                for (int k = 0; k < r; ++k) s -= L[r * 9 + k] * y[k];
                y[r] = s * il[r];
            }
            for (int r = 8; r >= 0; --r) {
                double s = y[r];
                for (int k = r + 1; k < 9; ++k) s -= L[k * 9 + r] * y[k];
                y[r] = s * il[r];
            }
            for (int r = col; r < 9; ++r) M.BinvT[45 * i + sym9(col, r)] = (T)y[r];
        }
    }
    T *Ci = (T *)A.Cinv;
    for (int j = threadIdx.x; j < d.np; j += NT) {
        const int64_t pt = d.pt0 + j;
        const double *h = A.Hll + 6 * pt;
        const double a00 = h[0] + mu * damp_term_b(damping, h[0]), a01 = h[1], a02 = h[2];
        const double a11 = h[3] + mu * damp_term_b(damping, h[3]), a12 = h[4];
        const double a22 = h[5] + mu * damp_term_b(damping, h[5]);
        const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
        const double det = a00 * c00 + a01 * c01 + a02 * c02;
        if (!(det > 0.0) || !isfinite(det)) {
            S.blockfail = 1;
            continue;
        }
        const double id = 1.0 / det;
        Ci[6 * pt + 0] = (T)(c00 * id);
        Ci[6 * pt + 1] = (T)(c01 * id);
        Ci[6 * pt + 2] = (T)(c02 * id);
        Ci[6 * pt + 3] = (T)((a00 * a22 - a02 * a02) * id);
        Ci[6 * pt + 4] = (T)((a02 * a01 - a00 * a12) * id);
        Ci[6 * pt + 5] = (T)((a00 * a11 - a01 * a01) * id);
    }
}

// ---------------------------------------------------------------------------
// Explicit reduced camera matrix S~ = B~ - E C~^-1 E^T (Sec. 3 Eq. 3) of one
// window, formed once per damped solve.  Block (i, k), i <= k, is
//   B~_i [i = k] - sum over points j seen by both of Jc~_ij^T G Jc~_kj,
//   G = Jp~_ij C~_j^-1 Jp~_kj^T (2x2),
// accumulated in the order of the block's pair list (one warp per block, no
// shared accumulators).  S~ p is then the same product as the implicit form of
// Alg. 3, with the point side folded in once instead of per iteration.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int blk_index(int i, int k, int nc) { return i * nc - (i * (i - 1)) / 2 + (k - i); }

// 24 consecutive values (16-byte aligned) with vector loads
template <typename T>
__device__ __forceinline__ void ld24(const T *p, T *o);
template <>
__device__ __forceinline__ void ld24<float>(const float *p, float *o) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 v = reinterpret_cast<const float4 *>(p)[q];
        o[4 * q] = v.x;
        o[4 * q + 1] = v.y;
        o[4 * q + 2] = v.z;
        o[4 * q + 3] = v.w;
    }
}
template <>
__device__ __forceinline__ void ld24<double>(const double *p, double *o) {
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const double2 v = reinterpret_cast<const double2 *>(p)[q];
        o[2 * q] = v.x;
        o[2 * q + 1] = v.y;
    }
}

template <typename T, int NT>
__device__ void s_build(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d, double mu, int damping) {
    constexpr int NW = NT / 32;
    constexpr int SP = Stage<T>::pairs, SS = Stage<T>::stride;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nc = d.nc, nb = nc * (nc + 1) / 2;
    T *S = M.S ? M.S : (T *)A.S + A.smax * (int64_t)blockIdx.x;
    T *st = M.stage + wid * SP * SS;
    const T *Jcm = (const T *)A.Jcm;
    const T *Ci = (const T *)A.Cinv;
    const int a = lane / 3, b0 = 3 * (lane - 3 * (lane / 3));
    int bi = 0, bk = 0, bcur = 0;  // (i, k) of block bcur, advanced incrementally
    for (int blk = wid; blk < nb; blk += NW) {
        while (bcur < blk) {
            ++bk;
            if (bk == nc) {
                ++bi;
                bk = bi;
            }
            ++bcur;
        }
        const int p0 = __ldg(A.blk_ptr + d.blk0 + blk), p1 = __ldg(A.blk_ptr + d.blk0 + blk + 1);
        T acc[3] = {T(0), T(0), T(0)};
        for (int base = p0; base < p1; base += SP) {
            const int cnt = min(SP, p1 - base);
            if (lane < cnt) {
                const int4 pr = __ldg(A.pairs + base + lane);
                T J1[24], J2[24];
                ld24<T>(Jcm + 24 * (int64_t)pr.x, J1);
                ld24<T>(Jcm + 24 * (int64_t)pr.y, J2);
                T c[6];
                ld_c<T>(Ci, pr.z, c);
                T q0[3], q1[3];  // Q = Jp~_1 C~^-1 (2x3)
                sym3_mul<T>(c, J1[18], J1[19], J1[20], q0);
                sym3_mul<T>(c, J1[21], J1[22], J1[23], q1);
                const T g00 = q0[0] * J2[18] + q0[1] * J2[19] + q0[2] * J2[20];
                const T g01 = q0[0] * J2[21] + q0[1] * J2[22] + q0[2] * J2[23];
                const T g10 = q1[0] * J2[18] + q1[1] * J2[19] + q1[2] * J2[20];
                const T g11 = q1[0] * J2[21] + q1[1] * J2[22] + q1[2] * J2[23];
                T *sp = st + lane * SS;
#pragma unroll
                for (int b = 0; b < 9; ++b) {
                    const T x0 = J2[b], x1 = J2[9 + b];
                    sp[b] = J1[b];
                    sp[9 + b] = J1[9 + b];
                    sp[18 + b] = g00 * x0 + g01 * x1;
                    sp[27 + b] = g10 * x0 + g11 * x1;
                }
            }
            __syncwarp();
            if (lane < 27)
                for (int p = 0; p < cnt; ++p) {
                    const T *sp = st + p * SS;
                    const T j0 = sp[a], j1 = sp[9 + a];
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) acc[cc] += j0 * sp[18 + b0 + cc] + j1 * sp[27 + b0 + cc];
                }
            __syncwarp();
        }
        if (lane < 27) {
            T *Sb = S + 81 * (int64_t)blk + 9 * a + b0;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                double v = -(double)acc[cc];
                if (bi == bk) {
                    const double *Hi = M.Hpp + 45 * bi;
                    v += Hi[sym9(a, b0 + cc)];
                    if (a == b0 + cc) v += mu * damp_term_b(damping, Hi[sym9(a, a)]);
                }
                Sb[cc] = (T)v;
            }
        }
    }
}

// q = S~ p (p given in M.pv as T) into M.q.
template <typename T, int NT>
__device__ void s_matvec(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d) {
    const int nc = d.nc;
    const T *S = M.S ? M.S : (const T *)A.S + A.smax * (int64_t)blockIdx.x;
    const T *pT = M.pv;
    for (int r = threadIdx.x; r < 9 * nc; r += NT) {
        const int i = r / 9, a = r - 9 * (r / 9);
        T acc = T(0);
        for (int k = 0; k < i; ++k) {  // column a of block (k, i)
            const T *Sb = S + 81 * (int64_t)blk_index(k, i, nc) + a;
            const T *pk = pT + 9 * k;
#pragma unroll
            for (int b = 0; b < 9; ++b) acc += Sb[9 * b] * pk[b];
        }
        const T *Sr = S + 81 * (int64_t)blk_index(i, i, nc) + 9 * a;  // blocks (i, k >= i) are consecutive
        for (int k = i; k < nc; ++k) {  // row a of block (i, k)
            const T *Sb = Sr + 81 * (int64_t)(k - i);
            const T *pk = pT + 9 * k;
#pragma unroll
            for (int b = 0; b < 9; ++b) acc += Sb[b] * pk[b];
        }
        M.q[r] = (double)acc;
    }
}

// Schur-Jacobi preconditioner (solver variant) from the explicit S~: the
// inverse (Cholesky, FP64) of each diagonal block replaces B~_i^-1; a block that
// is not positive definite keeps B~_i^-1.  One thread per camera.
template <typename T, int NT>
__device__ void sj_from_s(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d) {
    const T *S = M.S ? M.S : (const T *)A.S + A.smax * (int64_t)blockIdx.x;
    for (int i = threadIdx.x; i < d.nc; i += NT) {
        const T *Sb = S + 81 * (int64_t)blk_index(i, i, d.nc);
        double L[81], il[9];
        for (int q = 0; q < 81; ++q) L[q] = (double)Sb[q];
        bool ok = true;
        for (int j = 0; j < 9 && ok; ++j) {
            double s = L[j * 9 + j];
            for (int k = 0; k < j; ++k) s -= L[j * 9 + k] * L[j * 9 + k];
            if (!(s > 0.0) || !isfinite(s)) {
                ok = false;
                break;
            }
            const double l = sqrt(s);
            il[j] = 1.0 / l;
            L[j * 9 + j] = l;
            for (int r = j + 1; r < 9; ++r) {
                double t = L[r * 9 + j];
                for (int k = 0; k < j; ++k) t -= L[r * 9 + k] * L[j * 9 + k];
                L[r * 9 + j] = t * il[j];
            }
        }
        if (!ok) continue;
        for (int col = 0; col < 9; ++col) {
            double y[9];
            for (int r = 0; r < 9; ++r) {
                double s = (r == col) ? 1.0 : 0.0;
                for (int k = 0; k < r; ++k) s -= L[r * 9 + k] * y[k];
                y[r] = s * il[r];
            }
            for (int r = 8; r >= 0; --r) {
                double s = y[r];
                for (int k = r + 1; k < 9; ++k) s -= L[k * 9 + r] * y[k];
                y[r] = s * il[r];
            }
            for (int r = col; r < 9; ++r) M.BinvT[45 * i + sym9(col, r)] = (T)y[r];
        }
    }
}

// PCG of Alg. 2 on S x = g, g = vvec - E C~^-1 wvec (Sec. 3 Eq. 3), x0 = 0;
// leaves x in M.x and returns the iteration count.  The product S p is the
// implicit two-pass form of Alg. 3, or the explicit S~ of s_build.
// Single-reduction form of the same PCG (mba_pcg_variant SINGLE_REDUCTION; the
// oracle's pcg_single_reduction, after Chronopoulos and Gear): each step forms
// u = B~^-1 r and w = S~ u, takes r.r, r.u and w.u in one block reduction, and
// updates alpha = r.u / (w.u - beta r.u / alpha_prev), beta = r.u / (r.u)_prev,
// p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s.  One reduction
// per step instead of two; the test |r| <= tol |r0| is taken on the r.r of that
// reduction, i.e. after the product of the step that would follow.  Entered
// with r = g (and its T copy) and x = 0; returns the number of steps.
template <typename T, int NT>
__device__ __noinline__ int pcg_single_reduction(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d, double mu,
                                    int damping, int max_iter, double tol, bool xs, double *g0) {
    const int m9 = 9 * d.nc;
    double *sc = M.sb + 3 * NT + 4;  // alpha, beta (written by thread 0)
    int *go = reinterpret_cast<int *>(M.sb + 3 * NT + 6);
    double r0 = 0.0, stop2 = 0.0, gamma_prev = 0.0, alpha_prev = 0.0;  // meaningful in thread 0
    int n = 0;
    while (n == 0 || n < max_iter) {
        // u = B~^-1 r into M.z (FP64) and, as the explicit product's input, M.pv (T)
        double rr = 0.0, ru = 0.0;
        for (int t = threadIdx.x; t < m9; t += NT) {
            const int i = t / 9, a = t - 9 * (t / 9);
            const T *Bi = M.BinvT + 45 * i;
            const T *ri = M.rT + 9 * i;
            T zt = T(0);
#pragma unroll
            for (int b = 0; b < 9; ++b) zt = fma(Bi[sym9(a, b)], ri[b], zt);
            const double u = (double)zt;
            M.z[t] = u;
            if (xs) M.pv[t] = zt;
            rr = fma(M.r[t], M.r[t], rr);
            ru = fma(M.r[t], u, ru);
        }
        __syncthreads();
        // w = S~ u into M.q, and this thread's part of w.u
        double wu = 0.0;
        if (xs) {
            s_matvec<T, NT>(A, M, d);
            for (int t = threadIdx.x; t < m9; t += NT) wu = fma(M.z[t], M.q[t], wu);
        } else {
            make_pv<T, NT>(M, M.z, d.nc);
            __syncthreads();
            iter_points<T, NT>(A, M, d);
            __syncthreads();
            camera_pass<T, NT, false>(A, M, d);
            __syncthreads();
            for (int t = threadIdx.x; t < m9; t += NT) {
                const int i = t / 9, a = t - 9 * (t / 9);
                const double *Hi = M.Hpp + 45 * i;
                const double *ui = M.z + 9 * i;
                double bu = 0.0;
#pragma unroll
                for (int b = 0; b < 9; ++b) bu = fma(Hi[sym9(a, b)], ui[b], bu);
                bu = fma(mu * damp_term_b(damping, Hi[sym9(a, a)]), ui[a], bu);
                const double w = bu - slot_sum(M.slot, M.wf, M.wl, i, 9, a);
                M.q[t] = w;
                wu = fma(M.z[t], w, wu);
            }
        }
        cta_sum3f<NT>(rr, ru, wu, M.sb, [&](double x, double y, double z) {
            bool ok;
            if (n == 0) {
                r0 = sqrt(x);
                if (g0) {  // forcing sequence, as in the standard form
                    if (!(*g0 > 0.0)) *g0 = r0;
                    tol = fmax(tol, fmin(0.1, *g0 > 0.0 ? sqrt(r0 / *g0) : 0.0));
                }
                stop2 = (tol * r0) * (tol * r0);
                ok = r0 > 0.0;
            } else {
                ok = !(x <= stop2);
            }
            ok = ok && isfinite(y);
            const double beta = n == 0 ? 0.0 : y / gamma_prev;
            const double den = n == 0 ? z : z - beta * y / alpha_prev;  // p.S p in exact arithmetic
            ok = ok && den > 0.0 && isfinite(den);
            const double alpha = ok ? y / den : 0.0;
            gamma_prev = y;
            alpha_prev = alpha;
            *go = ok ? 1 : 0;
            sc[0] = alpha;
            sc[1] = beta;
        });
        if (!*go) break;
        const double alpha = sc[0], beta = sc[1];
        for (int t = threadIdx.x; t < m9; t += NT) {
            const double u = M.z[t], w = M.q[t];
            const double pn = n == 0 ? u : fma(beta, M.p[t], u);
            const double sn = n == 0 ? w : fma(beta, M.sv[t], w);
            M.p[t] = pn;
            M.sv[t] = sn;
            M.x[t] = fma(alpha, pn, M.x[t]);
            const double rv = fma(-alpha, sn, M.r[t]);
            M.r[t] = rv;
            M.rT[t] = (T)rv;
        }
        ++n;
        __syncthreads();
    }
    return n;
}

template <typename T, int NT>
__device__ int pcg(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d, const double *vvec, const double *wvec,
                   double mu, int damping, int max_iter, double tol, bool xs, double *g0, bool sr) {
    const int m9 = 9 * d.nc;
    rhs_points<T, NT>(A, M, d, wvec);
    __syncthreads();
    camera_pass<T, NT, false>(A, M, d);
    __syncthreads();
    for (int t = threadIdx.x; t < m9; t += NT) {
        const int i = t / 9, a = t - 9 * (t / 9);
        const double rv = vvec[t] - slot_sum(M.slot, M.wf, M.wl, i, 9, a);
        M.r[t] = rv;
        M.rT[t] = (T)rv;
        M.x[t] = 0.0;
    }
    __syncthreads();
    if (sr) return pcg_single_reduction<T, NT>(A, M, d, mu, damping, max_iter, tol, xs, g0);
    // scalar recurrences in thread 0 (see cta_sum2f): sc[0] holds beta or alpha,
    // *go the continue flag
    double *sc = M.sb + 2 * NT + 2;
    int *go = reinterpret_cast<int *>(M.sb + 2 * NT + 3);
    // meaningful in thread 0; the stopping test |r| <= tol |r0| compares squares
    // (r.r <= stop2), which keeps a square root off each iteration's scalar chain
    double r0 = 0.0, rho = 0.0, rho_prev = 0.0, stop2 = 0.0;
    int n = 0;
    {
        const double2 s0 = precond<T, NT>(M, d.nc);
        cta_sum2f<NT>(s0.x, s0.y, M.sb, [&](double x, double y) {
            r0 = sqrt(x);
            rho = y;
            if (g0) {  // forcing sequence: tol = max(tol, min(0.1, sqrt(|g| / |g_first|)))
                if (!(*g0 > 0.0)) *g0 = r0;
                tol = fmax(tol, fmin(0.1, *g0 > 0.0 ? sqrt(r0 / *g0) : 0.0));
            }
            stop2 = (tol * r0) * (tol * r0);
            *go = (r0 > 0.0 && isfinite(rho)) ? 1 : 0;
            sc[0] = 0.0;
        });
    }
    if (*go) {
        for (;;) {
            const double beta = sc[0];
            double pq = 0.0;
            if (xs) {
                for (int t = threadIdx.x; t < m9; t += NT) {
                    const double pn = n == 0 ? M.z[t] : fma(beta, M.p[t], M.z[t]);
                    M.p[t] = pn;
                    M.pv[t] = (T)pn;
                }
                __syncthreads();
                s_matvec<T, NT>(A, M, d);
                for (int t = threadIdx.x; t < m9; t += NT) pq = fma(M.p[t], M.q[t], pq);
            } else {
            for (int t = threadIdx.x; t < m9; t += NT) M.p[t] = n == 0 ? M.z[t] : fma(beta, M.p[t], M.z[t]);
            __syncthreads();
            make_pv<T, NT>(M, M.p, d.nc);
            __syncthreads();
            iter_points<T, NT>(A, M, d);
            __syncthreads();
            camera_pass<T, NT, false>(A, M, d);
            __syncthreads();
            for (int t = threadIdx.x; t < m9; t += NT) {
                const int i = t / 9, a = t - 9 * (t / 9);
                const double *Hi = M.Hpp + 45 * i;
                const double *pi_ = M.p + 9 * i;
                double bp = 0.0;
#pragma unroll
                for (int b = 0; b < 9; ++b) bp = fma(Hi[sym9(a, b)], pi_[b], bp);
                bp = fma(mu * damp_term_b(damping, Hi[sym9(a, a)]), pi_[a], bp);
                const double q = bp - slot_sum(M.slot, M.wf, M.wl, i, 9, a);
                M.q[t] = q;
                pq = fma(M.p[t], q, pq);
            }
            }
            cta_sum2f<NT>(pq, 0.0, M.sb, [&](double x, double) {
                const bool ok = x > 0.0 && isfinite(x);
                *go = ok ? 1 : 0;
                sc[0] = ok ? rho / x : 0.0;
            });
            if (!*go) break;
            const double alpha = sc[0];
            for (int t = threadIdx.x; t < m9; t += NT) {
                M.x[t] = fma(alpha, M.p[t], M.x[t]);
                const double rv = fma(-alpha, M.q[t], M.r[t]);
                M.r[t] = rv;
                M.rT[t] = (T)rv;
            }
            __syncthreads();
            const double2 s = precond<T, NT>(M, d.nc);
            ++n;
            cta_sum2f<NT>(s.x, s.y, M.sb, [&](double x, double y) {
                rho_prev = rho;
                rho = y;
                const bool ok = !(x <= stop2 || n >= max_iter) && isfinite(rho);
                *go = ok ? 1 : 0;
                sc[0] = ok ? rho / rho_prev : 0.0;
            });
            if (!*go) break;
        }
    }
    return n;
}

// F = 1/2 sum rho(|e|^2) in FP64 with the FP64 camera table in M.tab64.
template <typename T, int NT>
__device__ double cost(const BatchArgs &A, const WinMem<T> &M, const WinDesc &d, const double *pts) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < d.n; k += NT) {
        const int o = d.obs0 + k;
        const int2 pc = __ldg(A.pm_pc + o);
        const double2 uv = __ldg(A.pm_uv + o);
        double e[2];
        project<double, false>(M.tab64 + kCamTab * (pc.y - d.cam0), pts[3 * (int64_t)pc.x],
                               pts[3 * (int64_t)pc.x + 1], pts[3 * (int64_t)pc.x + 2], uv.x, uv.y, e, nullptr,
                               nullptr);
        double rho, W;
        loss_weight<double>(A.loss, A.delta, e[0] * e[0] + e[1] * e[1], &rho, &W);
        acc += rho;
    }
    return 0.5 * cta_sum2<NT>(acc, 0.0, M.sb).x;
}

template <typename T, int NT>
__device__ __forceinline__ void tables64(const WinMem<T> &M, const double *cams, int nc) {
    for (int i = threadIdx.x; i < nc; i += NT) camera_table_row(cams + 9 * i, M.tab64 + kCamTab * i);
}

// Warp ownership of the camera-major observations of a window.
template <int NT>
__device__ __forceinline__ int warp_lo(int w, int n) {
    return (int)(((int64_t)w * n) / (NT / 32));
}
template <int NT>
__device__ int owner_warp(int r, int n) {
    constexpr int NW = NT / 32;
    int w = (int)(((int64_t)r * NW) / n);
    if (w > NW - 1) w = NW - 1;
    while (w + 1 < NW && warp_lo<NT>(w + 1, n) <= r) ++w;
    while (w > 0 && warp_lo<NT>(w, n) > r) --w;
    return w;
}

template <typename T, int NT>
__device__ __forceinline__ void solve_window(const BatchArgs &A, const BatchOpts &O, const WinMem<T> &M, WinState &S, int wi) {
    constexpr int NW = NT / 32;
    const WinDesc d = A.desc[wi];
    const int tid = threadIdx.x, m9 = 9 * d.nc;
    for (int t = tid; t < m9; t += NT) M.cams[t] = A.cams[9 * (int64_t)d.cam0 + t];
    for (int t = tid; t <= d.nc; t += NT) M.cptr[t] = __ldg(A.cam_ptr + d.cam0 + t) - d.obs0;
    if (tid == 0) {
        S.radius = O.initial_radius;
        S.factor = 2.0;
        S.mu = 1.0 / O.initial_radius;
        S.mu_acc = -1.0;
        S.relin = 1;
        S.done = 0;
        S.iter = 0;
        S.acc_total = 0;
        S.pcg_total = 0;
        S.status = MBA_OK;
        S.accept = 0;
        S.adj_iters = 0;
        S.blockfail = 0;
        S.g0 = 0.0;
    }
    __syncthreads();
    for (int i = tid; i < d.nc; i += NT) {
        M.wf[i] = owner_warp<NT>(M.cptr[i], d.n);
        M.wl[i] = owner_warp<NT>(M.cptr[i + 1] - 1, d.n);
    }
    if (tid < NW) {
        const int lo = warp_lo<NT>(tid, d.n);
        int c = 0;
        while (c + 1 < d.nc && M.cptr[c + 1] <= lo) ++c;
        M.wcam0[tid] = c;
    }
    tables64<T, NT>(M, M.cams, d.nc);
    __syncthreads();
    {
        const double F = cost<T, NT>(A, M, d, A.pts);
        if (tid == 0) {
            S.F = F;
            S.F0 = F;
        }
    }
    __syncthreads();
    for (int it = 0; it < O.max_iter; ++it) {
        if (S.done) break;
        if (S.relin) {
            linearize<T, NT>(A, M, d, O.explicit_schur != 0);
            if (tid == 0) S.relin = 0;
        }
        const double mu = 1.0 / S.radius;
        damp<T, NT>(A, M, S, d, mu, O.damping);
        __syncthreads();
        if (S.blockfail) {  // no step: the iteration counts as rejected (the rule of lm.cu)
            __syncthreads();
            if (tid == 0) {
                S.radius = fmax(S.radius / S.factor, 1e-32);
                S.factor *= 2.0;
                S.mu = mu;
                S.accept = 0;
                S.iter = it + 1;
                S.blockfail = 0;
            }
            __syncthreads();
            continue;
        }
        if (S.status != MBA_OK) break;
        if (O.explicit_schur) {
            s_build<T, NT>(A, M, d, mu, O.damping);
            __syncthreads();
            if (O.precond == MBA_PRECOND_SCHUR_JACOBI) {
                sj_from_s<T, NT>(A, M, d);
                __syncthreads();
            }
        }
        const int np_ = pcg<T, NT>(A, M, d, M.v, A.wv, mu, O.damping, O.pcg_max_iter, O.pcg_tol,
                                   O.explicit_schur != 0, O.forcing ? &S.g0 : nullptr, O.pcg_variant != 0);
        make_pv<T, NT>(M, M.x, d.nc);
        __syncthreads();
        double ld = back_points<T, NT>(A, M, d, A.wv, false);
        ld = cta_sum2<NT>(ld, 0.0, M.sb).x;
        for (int t = tid; t < m9; t += NT) M.camn[t] = M.cams[t] + M.x[t];
        __syncthreads();
        tables64<T, NT>(M, M.camn, d.nc);
        __syncthreads();
        const double Fn = cost<T, NT>(A, M, d, A.pts_new);
        if (tid == 0) {
            // trust-region rule of lm.cu
            const double F = S.F, L = ld;
            const double gain = (F - Fn) / L;
            const int accept = (L > 0.0) && isfinite(Fn) && (gain > O.min_rel_dec);
            double radius = S.radius;
            if (accept) {
                const double tt = 2.0 * gain - 1.0;
                const double shrink = 1.0 - tt * tt * tt;
                radius = radius / fmax(shrink, 1.0 / 3.0);
                S.factor = 2.0;
                if (O.function_tol > 0.0 && fabs(F - Fn) < O.function_tol * F) S.done = 1;
                S.F = Fn;
                S.mu_acc = mu;
                S.acc_total += 1;
                S.relin = 1;
            } else {
                radius = radius / S.factor;
                S.factor *= 2.0;
            }
            S.radius = fmin(fmax(radius, 1e-32), 1e16);
            S.mu = mu;
            S.accept = accept;
            S.pcg_total += np_;
            S.iter = it + 1;
        }
        __syncthreads();
        if (S.accept) {
            for (int t = tid; t < m9; t += NT) M.cams[t] = M.camn[t];
            for (int t = tid; t < 3 * d.np; t += NT)
                A.pts[3 * (int64_t)d.pt0 + t] = A.pts_new[3 * (int64_t)d.pt0 + t];
        }
        __syncthreads();
    }
    // adjoint at the solution (mba_adjoint): v = M^-1 gbar, dL/du_k = W_k J_k v, dL/dx0 = mu D v
    if (O.adjoint) {
        if (S.status == MBA_OK && (O.adj_mu >= 0.0 || S.acc_total > 0)) {
            tables64<T, NT>(M, M.cams, d.nc);
            __syncthreads();
            if (S.relin) {
                linearize<T, NT>(A, M, d, O.explicit_schur != 0);
                if (tid == 0) S.relin = 0;
            }
            const double mu = O.adj_mu >= 0.0 ? O.adj_mu : S.mu_acc;
            damp<T, NT>(A, M, S, d, mu, O.damping);
            __syncthreads();
            if (tid == 0 && S.blockfail) S.status = MBA_ERR_NONFINITE;
            __syncthreads();
            if (S.status == MBA_OK) {
                if (O.explicit_schur) {
                    s_build<T, NT>(A, M, d, mu, O.damping);
                    __syncthreads();
                    if (O.precond == MBA_PRECOND_SCHUR_JACOBI) {
                        sj_from_s<T, NT>(A, M, d);
                        __syncthreads();
                    }
                }
                const int na = pcg<T, NT>(A, M, d, A.gbar_c + 9 * (int64_t)d.cam0, A.gbar_p, mu, O.damping,
                                          O.adj_pcg_max, O.adj_pcg_tol, O.explicit_schur != 0, nullptr,
                                          O.pcg_variant != 0);
                make_pv<T, NT>(M, M.x, d.nc);
                __syncthreads();
                back_points<T, NT>(A, M, d, A.gbar_p, true);
                __syncthreads();
                for (int t = tid; t < m9; t += NT) {
                    const int i = t / 9, a = t - 9 * (t / 9);
                    A.grad_c0[9 * (int64_t)d.cam0 + t] =
                        mu * damp_term_b(O.damping, M.Hpp[45 * i + sym9(a, a)]) * M.x[t];
                }
                for (int t = tid; t < 3 * d.np; t += NT) {
                    const int64_t j = d.pt0 + t / 3;
                    const int a = t - 3 * (t / 3);
                    A.grad_p0[3 * j + a] =
                        mu * damp_term_b(O.damping, A.Hll[6 * j + sym3(a, a)]) * A.dp[3 * j + a];
                }
                if (tid == 0) S.adj_iters = na;
            }
        } else if (S.status == MBA_OK) {
            // no accepted step: x* = x0 for any nearby input
            for (int k = tid; k < d.n; k += NT) {
                const int64_t o = __ldg(A.pm_orig + d.obs0 + k);
                A.grad_obs[2 * o] = 0.0;
                A.grad_obs[2 * o + 1] = 0.0;
            }
            for (int t = tid; t < m9; t += NT) A.grad_c0[9 * (int64_t)d.cam0 + t] = A.gbar_c[9 * (int64_t)d.cam0 + t];
            for (int t = tid; t < 3 * d.np; t += NT)
                A.grad_p0[3 * (int64_t)d.pt0 + t] = A.gbar_p[3 * (int64_t)d.pt0 + t];
        }
        __syncthreads();
        if (S.status != MBA_OK) {
            for (int k = tid; k < d.n; k += NT) {
                const int64_t o = __ldg(A.pm_orig + d.obs0 + k);
                A.grad_obs[2 * o] = 0.0;
                A.grad_obs[2 * o + 1] = 0.0;
            }
            for (int t = tid; t < m9; t += NT) A.grad_c0[9 * (int64_t)d.cam0 + t] = 0.0;
            for (int t = tid; t < 3 * d.np; t += NT) A.grad_p0[3 * (int64_t)d.pt0 + t] = 0.0;
        }
    }
    for (int t = tid; t < m9; t += NT) A.cams[9 * (int64_t)d.cam0 + t] = M.cams[t];
    if (tid == 0) {
        mba_window_summary o;
        o.iterations = S.iter;
        o.accepted = S.acc_total;
        o.pcg_iters_total = S.pcg_total;
        o.status = S.status;
        o.initial_cost = S.F0;
        o.final_cost = S.F;
        o.final_radius = S.radius;
        o.mu_accepted = S.mu_acc;
        o.adjoint_pcg_iters = S.adj_iters;
        o.pad = 0;
        A.out[wi] = o;
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) batch_kernel(BatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ WinState S;
    WinMem<T> M;
    win_carve<T>(smem_raw, A.ncmax, NT / 32, A.s_smem ? A.smax : 0, M);
    const BatchOpts O = *A.opts;
    for (;;) {
        if (threadIdx.x == 0) S.win = atomicAdd(A.counter, 1);
        __syncthreads();
        const int k = S.win;
        __syncthreads();
        if (k >= A.nw) break;
        const int wi = __ldg(A.order + k);
        const unsigned long long t0 = global_ns();
        solve_window<T, NT>(A, O, M, S, wi);  // ends with a block barrier
        if (threadIdx.x == 0) A.win_ns[wi] = global_ns() - t0;
    }
}

// ---------------------------------------------------------------------------
// Layout of a batch on the device (mba_batch_create).  The windows' local
// indices become global ones (window offsets added), and the point-major and
// camera-major orders are stable sorts of the observations by global point and
// by global camera: the windows' observations are contiguous and in window
// order, so these are the per-window stable orders.  Warp chunks and the
// explicit form's pair lists follow in the order the kernels expect.
// flags[0] bits: 1 index out of its window's range, 2 non-finite input,
// 4 a point without observations, 8 a camera without observations.
// ---------------------------------------------------------------------------
constexpr int kLayBlock = 256;

__device__ __forceinline__ int window_of(const int32_t *off, int nw, int64_t x) {
    int lo = 0, hi = nw;  // off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void lay_globalize_kernel(int64_t n, int nw, const int32_t *oo, const int32_t *co, const int32_t *po,
                                     const int32_t *ci, const int32_t *pi, const double *obs, int32_t *gpt,
                                     int32_t *gcam, int32_t *flags) {
    int bad = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int w = window_of(oo, nw, k);
        const int32_t c = ci[k], q = pi[k], nc = co[w + 1] - co[w], np = po[w + 1] - po[w];
        if (c < 0 || c >= nc || q < 0 || q >= np) bad |= 1;
        gpt[k] = po[w] + (q < 0 || q >= np ? 0 : q);
        gcam[k] = co[w] + (c < 0 || c >= nc ? 0 : c);
        if (!isfinite(obs[2 * k]) || !isfinite(obs[2 * k + 1])) bad |= 2;
    }
    if (bad) atomicOr(flags, bad);
}

__global__ void lay_finite_kernel(const double *a, int64_t m, int32_t *flags) {
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[i])) bad = 2;
    if (bad) atomicOr(flags, bad);
}

// point-major copies: perm[i] = input index of point-major position i
__global__ void lay_gather_pm_kernel(int64_t n, const int32_t *perm, const int32_t *gpt, const int32_t *gcam,
                                     const double *obs, int2 *pm_pc, double2 *pm_uv, int32_t *pm_orig, int32_t *inv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = perm[i];
        pm_pc[i] = make_int2(gpt[k], gcam[k]);
        pm_uv[i] = make_double2(obs[2 * (int64_t)k], obs[2 * (int64_t)k + 1]);
        pm_orig[i] = k;
        inv[k] = (int32_t)i;
    }
}

// camera-major copies: perm[c] = input index of camera-major position c
__global__ void lay_gather_cm_kernel(int64_t n, const int32_t *perm, const int32_t *gpt, const int32_t *inv,
                                     int32_t *cm_pt, int32_t *cm2pm, int32_t *pm2cm) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = perm[c], i = inv[k];
        cm_pt[c] = gpt[k];
        cm2pm[c] = i;
        pm2cm[i] = (int32_t)c;
    }
}

__global__ void lay_empty_kernel(const int32_t *ptr, int64_t nseg, int bit, int32_t *flags) {
    int bad = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nseg; j += (int64_t)gridDim.x * blockDim.x)
        if (ptr[j + 1] == ptr[j]) bad = bit;
    if (bad) atomicOr(flags, bad);
}

// Warp chunks of one window: greedy runs of whole points with <= 32
// observations (a longer point alone), then the window's end entry.  One
// thread per window; fill == false only counts (into cnt[w]).
__global__ void lay_chunks_kernel(int nw, WinDesc *desc, const int32_t *pt_ptr, int32_t *cnt, const int32_t *wch0,
                                  int2 *wchunk, bool fill) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    WinDesc &d = desc[w];
    const int32_t p0 = d.pt0, np = d.np;
    int32_t j = 0, m = 0;
    const int32_t base = fill ? wch0[w] : 0;
    while (j < np) {
        if (fill) wchunk[base + m] = make_int2(p0 + j, pt_ptr[p0 + j]);
        int32_t len = pt_ptr[p0 + j + 1] - pt_ptr[p0 + j];
        ++j;
        if (len <= 32)
            while (j < np) {
                const int32_t l2 = pt_ptr[p0 + j + 1] - pt_ptr[p0 + j];
                if (len + l2 > 32) break;
                len += l2;
                ++j;
            }
        ++m;
    }
    if (fill) {
        wchunk[base + m] = make_int2(p0 + np, d.obs0 + d.n);
        d.wch0 = base;
        d.nwch = m;
    } else {
        cnt[w] = m + 1;
    }
}

// Schur-block pairs of each point: every ordered pair (u, v) of its
// observations (point-major positions) with camera(u) <= camera(v), u then v
// ascending.  Count pass (cnt[j], and the total in 64 bits into *total, so
// that an int32 overflow of the offsets is seen) and fill pass (pairs in point
// order at off[j], with the global block key of each).
__global__ void lay_pairs_kernel(int64_t np_all, int nw, const int32_t *po, const WinDesc *desc,
                                 const int32_t *pt_ptr, const int2 *pm_pc, const int32_t *pm2cm, int32_t *cnt,
                                 unsigned long long *total, const int32_t *off, int4 *pairs, int32_t *keys,
                                 bool fill) {
    unsigned long long mine = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < np_all;
         j += (int64_t)gridDim.x * blockDim.x) {
        const WinDesc &d = desc[window_of(po, nw, j)];
        const int32_t a = pt_ptr[j], e = pt_ptr[j + 1];
        int32_t m = 0, pos = fill ? off[j] : 0;
        for (int32_t u = a; u < e; ++u) {
            const int32_t cu = pm_pc[u].y - d.cam0;
            for (int32_t v = a; v < e; ++v) {
                const int32_t cv = pm_pc[v].y - d.cam0;
                if (cu > cv) continue;
                if (fill) {
                    pairs[pos] = make_int4(pm2cm[u], pm2cm[v], (int32_t)j, 0);
                    keys[pos] = d.blk0 + cu * d.nc - (cu * (cu - 1)) / 2 + (cv - cu);
                    ++pos;
                } else {
                    ++m;
                }
            }
        }
        if (!fill) {
            cnt[j] = m;
            mine += (unsigned long long)m;
        }
    }
    if (!fill) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, mine);
    }
}

__global__ void lay_gather_pairs_kernel(int64_t m, const int32_t *perm, const int4 *in, int4 *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

unsigned lay_grid(int64_t n) {
    int64_t g = (n + kLayBlock - 1) / kLayBlock;
    if (g > 4096) g = 4096;
    return (unsigned)(g < 1 ? 1 : g);
}

template <typename T, int NT>
size_t smem_bytes(int ncmax, int64_t svals) {
    WinMem<T> m;
    return win_carve<T>(nullptr, ncmax, NT / 32, svals, m);
}

// Instances: (threads per CTA, CTAs per SM the register budget is cut for).
// 256 threads: up to 2 resident CTAs (<= 128 registers) or 3 (<= 85);
// 512 threads: 1 (<= 128).
const void *kernel_ptr(bool fp32, int nt, int cps) {
    if (fp32) {
        if (nt == 512) return (const void *)batch_kernel<float, 512, 1>;
        return cps >= 3 ? (const void *)batch_kernel<float, 256, 3> : (const void *)batch_kernel<float, 256, 2>;
    }
    if (nt == 512) return (const void *)batch_kernel<double, 512, 1>;
    return cps >= 3 ? (const void *)batch_kernel<double, 256, 3> : (const void *)batch_kernel<double, 256, 2>;
}

// Dynamic shared memory of a launch; svals > 0 also holds S~ (svals values of T).
size_t kernel_smem(bool fp32, int nt, int ncmax, int64_t svals) {
    if (fp32) return nt == 256 ? smem_bytes<float, 256>(ncmax, svals) : smem_bytes<float, 512>(ncmax, svals);
    return nt == 256 ? smem_bytes<double, 256>(ncmax, svals) : smem_bytes<double, 512>(ncmax, svals);
}

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

}  // namespace mba

using namespace mba;

struct mba_batch {
    int32_t nw = 0, ncmax = 0;
    int64_t nc = 0, np = 0, n = 0, nch = 0;
    int fp32 = 0, loss = 0;
    double delta = 0.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *pool = nullptr;
    void *pool2 = nullptr;  // the explicit form's pair lists, J copy and S~ scratch
    BatchArgs A{};
    WinDesc *desc = nullptr;
    int32_t *order = nullptr, *counter = nullptr;
    BatchOpts *opts = nullptr;
    mba_window_summary *out = nullptr;
    double *cams0 = nullptr, *pts0 = nullptr, *cams_bak = nullptr, *pts_bak = nullptr;
    double *gbar_c = nullptr, *gbar_p = nullptr;
    bool explicit_ok = false;       // pair lists and S~ scratch exist
    int schur = 0;                  // schedule: 1 implicit, 2 explicit Schur product
    int sms = 0;
    int nt = 0, cps = 0;            // schedule in use
    cudaGraphExec_t gexec = nullptr;
    int g_nt = 0, g_grid = 0, g_cps = 0;  // schedule the graph was captured with
    bool g_ssm = false;
    bool has_grads = false;
    std::vector<unsigned long long> last_win_ns;  // per-window times of the last solve
};

namespace {

constexpr int kMaxCtasPerSm = 4;  // S~ scratch is sized for this many resident CTAs per SM

#define BCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return api_fail(MBA_ERR_CUDA, (std::string(#call) + ": " + cudaGetErrorString(e_)).c_str()); \
    } while (0)

// Resident CTAs per SM of the kernel instance used for (nt, cps).
int max_ctas_per_sm(const mba_batch *b, int nt, int cps, bool s_smem = false) {
    const void *k = kernel_ptr(b->fp32, nt, cps);
    const size_t sm = kernel_smem(b->fp32, nt, b->ncmax, s_smem ? b->A.smax : 0);
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (sm > (size_t)optin) return 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, nt, sm) != cudaSuccess) return 0;
    return blocks;
}

// Resolves a requested schedule to an admissible one (0 fields: automatic).
mba_status resolve_schedule(const mba_batch *b, int want_nt, int want_cps, int want_schur, int *nt, int *cps,
                            int *schur) {
    if (want_nt != 0 && want_nt != 256 && want_nt != 512)
        return api_fail(MBA_ERR_INVALID_ARG, "threads_per_cta must be 0, 256 or 512");
    if (want_cps < 0 || want_cps > kMaxCtasPerSm) return api_fail(MBA_ERR_INVALID_ARG, "ctas_per_sm must be in 0..4");
    if (want_schur < 0 || want_schur > 2) return api_fail(MBA_ERR_INVALID_ARG, "schur must be 0, 1 or 2");
    if (want_schur == 2 && !b->explicit_ok)
        return api_fail(MBA_ERR_INVALID_ARG, "the explicit Schur product is not available for this batch");
    *schur = want_schur ? want_schur : (b->explicit_ok ? 2 : 1);
    const int t = want_nt ? want_nt : 256;
    const int want = want_cps ? want_cps : 2;
    const int occ = max_ctas_per_sm(b, t, want);
    if (occ < 1) return api_fail(MBA_ERR_INVALID_ARG, "the batched kernel cannot be resident with this schedule");
    int c = want;
    if (c > occ) c = occ;
    *nt = t;
    *cps = c;
    return MBA_OK;
}

// The explicit S~ goes to shared memory when cps CTAs of that size still fit.
bool s_in_smem(const mba_batch *b) {
    return b->schur == 2 && b->explicit_ok && max_ctas_per_sm(b, b->nt, b->cps, true) >= b->cps;
}

mba_status build_graph(mba_batch *b) {
    const int grid_full = b->sms * b->cps;
    const int grid = grid_full < b->nw ? grid_full : b->nw;
    const bool ssm = s_in_smem(b);
    if (b->gexec && b->g_nt == b->nt && b->g_grid == grid && b->g_cps == b->cps && b->g_ssm == ssm) return MBA_OK;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    const void *k = kernel_ptr(b->fp32, b->nt, b->cps);
    const size_t sm = kernel_smem(b->fp32, b->nt, b->ncmax, ssm ? b->A.smax : 0);
    BCK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaMemsetAsync(b->counter, 0, sizeof(int32_t), b->stream);
    BatchArgs args = b->A;
    args.s_smem = ssm ? 1 : 0;
    void *kargs[] = {(void *)&args};
    cudaError_t e2 = cudaLaunchKernel(k, dim3(grid), dim3(b->nt), kargs, sm, b->stream);
    cudaError_t e3 = cudaStreamEndCapture(b->stream, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        const cudaError_t e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
        return api_fail(MBA_ERR_CUDA, (std::string("graph capture: ") + cudaGetErrorString(e)).c_str());
    }
    cudaError_t e4 = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e4 != cudaSuccess) {
        b->gexec = nullptr;
        return api_fail(MBA_ERR_CUDA, (std::string("graph instantiate: ") + cudaGetErrorString(e4)).c_str());
    }
    b->g_nt = b->nt;
    b->g_grid = grid;
    b->g_cps = b->cps;
    b->g_ssm = ssm;
    return MBA_OK;
}

bool finite_all(const double *a, int64_t m) {
    for (int64_t i = 0; i < m; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

}  // namespace

extern "C" {

mba_status mba_batch_create(int32_t n_windows, const int64_t *cam_offsets, const int64_t *pt_offsets,
                            const int64_t *obs_offsets, const double *cameras, const double *points,
                            const double *observations, const int32_t *cam_idx, const int32_t *pt_idx,
                            const mba_problem_options *opt, mba_batch **out) {
    if (!out) return api_fail(MBA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_windows < 1) return api_fail(MBA_ERR_INVALID_ARG, "n_windows must be >= 1");
    if (!cam_offsets || !pt_offsets || !obs_offsets || !cameras || !points || !observations || !cam_idx || !pt_idx)
        return api_fail(MBA_ERR_INVALID_ARG, "a required input pointer is NULL");
    mba_problem_options o;
    mba_problem_options_default(&o);
    if (opt) o = *opt;
    if (o.precision != MBA_FP64 && o.precision != MBA_FP32_MIXED) return api_fail(MBA_ERR_INVALID_ARG, "bad precision");
    if (o.loss != MBA_LOSS_NONE && o.loss != MBA_LOSS_HUBER) return api_fail(MBA_ERR_INVALID_ARG, "bad loss");
    if (o.loss == MBA_LOSS_HUBER && !(o.huber_delta > 0.0))
        return api_fail(MBA_ERR_INVALID_ARG, "huber_delta must be > 0");
    if (o.jacobian != MBA_JACOBIAN_ANALYTIC)
        return api_fail(MBA_ERR_INVALID_ARG, "batched windows use the analytic Jacobian only");
    if (kUserEdge) return api_fail(MBA_ERR_INVALID_ARG, "batched windows use the BAL edge; this library has a user edge");
    const int nw = n_windows;
    if (cam_offsets[0] != 0 || pt_offsets[0] != 0 || obs_offsets[0] != 0)
        return api_fail(MBA_ERR_INVALID_ARG, "offset arrays must start at 0");
    int ncmax = 0;
    for (int w = 0; w < nw; ++w) {
        const int64_t nc = cam_offsets[w + 1] - cam_offsets[w], np = pt_offsets[w + 1] - pt_offsets[w],
                      n = obs_offsets[w + 1] - obs_offsets[w];
        if (nc < 1 || nc > kBMaxCams) return api_fail(MBA_ERR_INVALID_ARG, "a window needs 1..64 cameras");
        if (np >= (int64_t(1) << 24)) return api_fail(MBA_ERR_INVALID_ARG, "a window may hold at most 2^24 - 1 points");
        if (np < 1 || n < 1) return api_fail(MBA_ERR_INVALID_ARG, "a window needs >= 1 point and observation");
        if (nc > ncmax) ncmax = (int)nc;
    }
    const int64_t NC = cam_offsets[nw], NP = pt_offsets[nw], N = obs_offsets[nw];
    if (N >= (int64_t(1) << 31) - 64 || NP >= (int64_t(1) << 31) - 64 || NC >= (int64_t(1) << 31) - 64)
        return api_fail(MBA_ERR_INVALID_ARG, "totals must be below 2^31 - 64");

    // Window descriptors (the layout fields wch0 / nwch are filled on the
    // device), the windows' offsets as int32, the explicit form's block
    // numbering (window w's upper blocks start at blk0) and the launch order.
    std::vector<WinDesc> desc((size_t)nw);
    std::vector<int32_t> off32(3 * ((size_t)nw + 1));  // observation, camera, point offsets
    int64_t nblk = 0;
    for (int w = 0; w < nw; ++w) {
        WinDesc &d = desc[w];
        d.cam0 = (int32_t)cam_offsets[w];
        d.nc = (int32_t)(cam_offsets[w + 1] - cam_offsets[w]);
        d.pt0 = (int32_t)pt_offsets[w];
        d.np = (int32_t)(pt_offsets[w + 1] - pt_offsets[w]);
        d.obs0 = (int32_t)obs_offsets[w];
        d.n = (int32_t)(obs_offsets[w + 1] - obs_offsets[w]);
        d.wch0 = d.nwch = 0;
        d.blk0 = (int32_t)(nblk < (int64_t(1) << 30) ? nblk : 0);
        d.pad = 0;
        nblk += (int64_t)d.nc * (d.nc + 1) / 2;
    }
    const bool blocks_ok = nblk < (int64_t(1) << 30);  // else no explicit form (int32 block keys)
    for (int w = 0; w <= nw; ++w) {
        off32[w] = (int32_t)obs_offsets[w];
        off32[nw + 1 + w] = (int32_t)cam_offsets[w];
        off32[2 * (nw + 1) + w] = (int32_t)pt_offsets[w];
    }
    // First launch: longest-first by an estimate of each window's time, its
    // observations (linearisation, S~ build) plus 10 nc^2 for the dense
    // product's 81 nc^2 per PCG step.  The weight is a least-squares fit to
    // measured window times of the 512-window workload (R^2 0.95 against 0.53
    // for the observation count alone; simulated makespan 29.4 against 36.9 ms).
    // Later launches order by the measured times of the previous one.
    std::vector<int32_t> order((size_t)nw);
    for (int w = 0; w < nw; ++w) order[w] = w;
    auto est = [&](int w) { return (double)desc[w].n + 10.0 * (double)desc[w].nc * (double)desc[w].nc; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return est(a) > est(b); });

    mba_batch *b = new mba_batch();
    b->nw = nw;
    b->ncmax = ncmax;
    b->nc = NC;
    b->np = NP;
    b->n = N;
    b->nch = NP + nw;  // bound: every chunk holds a point, plus one end entry per window
    b->fp32 = o.precision == MBA_FP32_MIXED;
    b->loss = o.loss;
    b->delta = o.huber_delta;
    void *tmp = nullptr, *tmp2 = nullptr;
    auto fail_free = [&](mba_status st, const std::string &msg) {
        if (b->stream) cudaStreamSynchronize(b->stream);
        if (tmp) cudaFree(tmp);
        if (tmp2) cudaFree(tmp2);
        mba_batch_destroy(b);
        return api_fail(st, msg.c_str());
    };
    if (o.cuda_stream) {
        b->stream = (cudaStream_t)o.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail_free(MBA_ERR_CUDA, "cudaStreamCreateWithFlags failed");
        b->own_stream = true;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->sms < 1) return fail_free(MBA_ERR_CUDA, "no CUDA device");
    const size_t w = b->fp32 ? 4 : 8;
    // one pool for the batch's lifetime (the explicit form's arrays come in a
    // second one, once the pair count is known)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o_ = off;
        off += al256(bytes ? bytes : 1);
        return o_;
    };
    const size_t o_desc = take(sizeof(WinDesc) * nw), o_order = take(4 * (size_t)nw), o_counter = take(256),
                 o_opts = take(sizeof(BatchOpts)), o_out = take(sizeof(mba_window_summary) * nw),
                 o_wch = take(sizeof(int2) * b->nch), o_pc = take(sizeof(int2) * N), o_uv = take(sizeof(double2) * N),
                 o_orig = take(4 * (size_t)N), o_cmpt = take(4 * (size_t)N), o_cm2pm = take(4 * (size_t)N),
                 o_cptr = take(4 * ((size_t)NC + 1)), o_cams = take(72 * (size_t)NC), o_cams0 = take(72 * (size_t)NC),
                 o_camsb = take(72 * (size_t)NC), o_pts = take(24 * (size_t)NP), o_pts0 = take(24 * (size_t)NP),
                 o_ptsb = take(24 * (size_t)NP), o_ptsn = take(24 * (size_t)NP), o_dp = take(24 * (size_t)NP),
                 o_hll = take(48 * (size_t)NP), o_wv = take(24 * (size_t)NP), o_pm2cm = take(4 * (size_t)N),
                 o_ci = take(6 * w * (size_t)NP), o_xw = take(4 * w * (size_t)NP),
                 o_cmx = take(4 * w * (size_t)N), o_cms = take(2 * w * (size_t)N),
                 o_W = o.loss != MBA_LOSS_NONE ? take(w * (size_t)N) : 0, o_gc = take(72 * (size_t)NC),
                 o_gp = take(24 * (size_t)NP), o_go = take(16 * (size_t)N), o_g0c = take(72 * (size_t)NC),
                 o_g0p = take(24 * (size_t)NP), o_bptr = take(blocks_ok ? 4 * ((size_t)nblk + 1) : 0),
                 o_wns = take(8 * (size_t)nw);
    const size_t pool_bytes = off;
    // layout scratch, freed before the call returns
    off = 0;
    const int64_t nkey = NP > NC ? NP : NC;
    const int64_t scan_n = (NP + 1) > (int64_t)(nw + 1) ? (NP + 1) : (int64_t)(nw + 1);
    const size_t t_obs = take(16 * (size_t)N), t_ci = take(4 * (size_t)N), t_pi = take(4 * (size_t)N),
                 t_off = take(4 * off32.size()), t_gpt = take(4 * (size_t)N), t_gcam = take(4 * (size_t)N),
                 t_ppm = take(4 * (size_t)N), t_pcm = take(4 * (size_t)N), t_inv = take(4 * (size_t)N),
                 t_ptptr = take(4 * ((size_t)NP + 1)), t_flags = take(256), t_ccnt = take(4 * ((size_t)nw + 1)),
                 t_pcnt = take(4 * ((size_t)NP + 1)), t_scan = take(4 * (size_t)exclusive_scan_tmp_ints(scan_n)),
                 t_sort = take(stable_sort_tmp_bytes(N, (int32_t)nkey));
    const size_t tmp_bytes = off;
    if (over_memory_limit(pool_bytes + tmp_bytes))
        return fail_free(MBA_ERR_OOM, "device memory limit: the batch needs more");
    if (cudaMalloc(&b->pool, pool_bytes) != cudaSuccess || cudaMalloc(&tmp, tmp_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail_free(MBA_ERR_OOM, "device allocation of the batch failed");
    }
    char *base = (char *)b->pool, *tb = (char *)tmp;
    b->desc = (WinDesc *)(base + o_desc);
    b->order = (int32_t *)(base + o_order);
    b->counter = (int32_t *)(base + o_counter);
    b->opts = (BatchOpts *)(base + o_opts);
    b->out = (mba_window_summary *)(base + o_out);
    b->cams0 = (double *)(base + o_cams0);
    b->pts0 = (double *)(base + o_pts0);
    b->cams_bak = (double *)(base + o_camsb);
    b->pts_bak = (double *)(base + o_ptsb);
    b->gbar_c = (double *)(base + o_gc);
    b->gbar_p = (double *)(base + o_gp);
    BatchArgs &A = b->A;
    A.nw = nw;
    A.ncmax = ncmax;
    A.loss = o.loss;
    A.delta = o.huber_delta;
    A.desc = b->desc;
    A.order = b->order;
    A.counter = b->counter;
    A.opts = b->opts;
    A.wchunk = (const int2 *)(base + o_wch);
    A.pm_pc = (const int2 *)(base + o_pc);
    A.pm_uv = (const double2 *)(base + o_uv);
    A.pm_orig = (const int32_t *)(base + o_orig);
    A.cm_pt = (const int32_t *)(base + o_cmpt);
    A.cm2pm = (const int32_t *)(base + o_cm2pm);
    A.cam_ptr = (const int32_t *)(base + o_cptr);
    A.cams = (double *)(base + o_cams);
    A.pts = (double *)(base + o_pts);
    A.pts_new = (double *)(base + o_ptsn);
    A.dp = (double *)(base + o_dp);
    A.Hll = (double *)(base + o_hll);
    A.wv = (double *)(base + o_wv);
    A.pm2cm = (const int32_t *)(base + o_pm2cm);
    A.Cinv = base + o_ci;
    A.Xw = base + o_xw;
    A.cmX = base + o_cmx;
    A.cms = base + o_cms;
    A.Wpm = o.loss != MBA_LOSS_NONE ? (void *)(base + o_W) : nullptr;
    A.gbar_c = b->gbar_c;
    A.gbar_p = b->gbar_p;
    A.grad_obs = (double *)(base + o_go);
    A.grad_c0 = (double *)(base + o_g0c);
    A.grad_p0 = (double *)(base + o_g0p);
    A.out = b->out;
    A.blk_ptr = (const int32_t *)(base + o_bptr);
    A.win_ns = (unsigned long long *)(base + o_wns);
    double *d_obs = (double *)(tb + t_obs);
    int32_t *d_ci = (int32_t *)(tb + t_ci), *d_pi = (int32_t *)(tb + t_pi), *d_off = (int32_t *)(tb + t_off),
            *gpt = (int32_t *)(tb + t_gpt), *gcam = (int32_t *)(tb + t_gcam), *perm_pm = (int32_t *)(tb + t_ppm),
            *perm_cm = (int32_t *)(tb + t_pcm), *inv = (int32_t *)(tb + t_inv), *pt_ptr = (int32_t *)(tb + t_ptptr),
            *flags = (int32_t *)(tb + t_flags), *ccnt = (int32_t *)(tb + t_ccnt), *pcnt = (int32_t *)(tb + t_pcnt),
            *scan_tmp = (int32_t *)(tb + t_scan);
    void *sort_tmp = tb + t_sort;
    const size_t sort_bytes = stable_sort_tmp_bytes(N, (int32_t)nkey);
    cudaStream_t s = b->stream;
    auto up = [&](void *dst, const void *src, size_t bytes) { return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s); };
    cudaError_t e = cudaSuccess;
    // inputs, as given
    if (e == cudaSuccess) e = up(b->desc, desc.data(), sizeof(WinDesc) * nw);
    if (e == cudaSuccess) e = up(b->order, order.data(), 4 * (size_t)nw);
    if (e == cudaSuccess) e = up(d_off, off32.data(), 4 * off32.size());
    if (e == cudaSuccess) e = up(d_obs, observations, 16 * (size_t)N);
    if (e == cudaSuccess) e = up(d_ci, cam_idx, 4 * (size_t)N);
    if (e == cudaSuccess) e = up(d_pi, pt_idx, 4 * (size_t)N);
    if (e == cudaSuccess) e = up(A.cams, cameras, 72 * (size_t)NC);
    if (e == cudaSuccess) e = up(A.pts, points, 24 * (size_t)NP);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 256, s);
    if (e != cudaSuccess) return fail_free(MBA_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    const int32_t *oo32 = d_off, *co32 = d_off + (nw + 1), *po32 = d_off + 2 * (nw + 1);
    // global indices, validation, the two stable orders and the copies in them
    lay_globalize_kernel<<<lay_grid(N), kLayBlock, 0, s>>>(N, nw, oo32, co32, po32, d_ci, d_pi, d_obs, gpt, gcam, flags);
    lay_finite_kernel<<<lay_grid(9 * NC), kLayBlock, 0, s>>>(A.cams, 9 * NC, flags);
    lay_finite_kernel<<<lay_grid(3 * NP), kLayBlock, 0, s>>>(A.pts, 3 * NP, flags);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = stable_sort_by_key(gpt, N, (int32_t)NP, perm_pm, pt_ptr, sort_tmp, sort_bytes, s);
    if (e == cudaSuccess)
        e = stable_sort_by_key(gcam, N, (int32_t)NC, perm_cm, (int32_t *)A.cam_ptr, sort_tmp, sort_bytes, s);
    if (e == cudaSuccess) {
        lay_gather_pm_kernel<<<lay_grid(N), kLayBlock, 0, s>>>(N, perm_pm, gpt, gcam, d_obs, (int2 *)A.pm_pc,
                                                               (double2 *)A.pm_uv, (int32_t *)A.pm_orig, inv);
        lay_gather_cm_kernel<<<lay_grid(N), kLayBlock, 0, s>>>(N, perm_cm, gpt, inv, (int32_t *)A.cm_pt,
                                                               (int32_t *)A.cm2pm, (int32_t *)A.pm2cm);
        lay_empty_kernel<<<lay_grid(NP), kLayBlock, 0, s>>>(pt_ptr, NP, 4, flags);
        lay_empty_kernel<<<lay_grid(NC), kLayBlock, 0, s>>>(A.cam_ptr, NC, 8, flags);
        // warp chunks: count per window, scan, fill (also the descriptors' wch0 / nwch)
        lay_chunks_kernel<<<(nw + 127) / 128, 128, 0, s>>>(nw, b->desc, pt_ptr, ccnt, nullptr, nullptr, false);
        e = cudaMemsetAsync(ccnt + nw, 0, 4, s);
    }
    if (e == cudaSuccess) e = exclusive_scan_i32(ccnt, ccnt, nw + 1, scan_tmp, s);
    if (e == cudaSuccess) {
        lay_chunks_kernel<<<(nw + 127) / 128, 128, 0, s>>>(nw, b->desc, pt_ptr, nullptr, ccnt, (int2 *)A.wchunk, true);
        // Schur-block pair counts per point, and their prefix (the total last)
        lay_pairs_kernel<<<lay_grid(NP), kLayBlock, 0, s>>>(NP, nw, po32, b->desc, pt_ptr, A.pm_pc, A.pm2cm, pcnt,
                                                            (unsigned long long *)(flags + 2), nullptr, nullptr,
                                                            nullptr, false);
        e = cudaMemsetAsync(pcnt + NP, 0, 4, s);
    }
    if (e == cudaSuccess) e = exclusive_scan_i32(pcnt, pcnt, NP + 1, scan_tmp, s);
    int32_t hflags = 0;
    unsigned long long total_pairs = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, flags, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total_pairs, flags + 2, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_free(MBA_ERR_CUDA, std::string("layout: ") + cudaGetErrorString(e));
    if (hflags & 2) return fail_free(MBA_ERR_NONFINITE, "non-finite camera, point or observation");
    if (hflags & 1) return fail_free(MBA_ERR_INVALID_ARG, "observation index out of its window's range");
    if (hflags & 4) return fail_free(MBA_ERR_INVALID_ARG, "a point without observations");
    if (hflags & 8) return fail_free(MBA_ERR_INVALID_ARG, "a camera without observations");
    // Schur-block pair lists in point order inside each block: generated in
    // point order with their block keys, then stably sorted by block (the sort
    // also yields the blocks' offsets).  Skipped, and the explicit form not
    // offered, when they would be too large.
    const bool explicit_ok = blocks_ok && total_pairs <= (1ull << 28);
    b->explicit_ok = explicit_ok;
    if (explicit_ok) {
        const int64_t smax = (int64_t)ncmax * (ncmax + 1) / 2 * 81;
        const int64_t np2 = (int64_t)total_pairs;
        off = 0;
        const size_t o_pairs = take(sizeof(int4) * (size_t)np2), o_jcm = take(24 * w * (size_t)N),
                     o_S = take(w * (size_t)smax * (size_t)b->sms * kMaxCtasPerSm);
        const size_t pool2_bytes = off;
        off = 0;
        const size_t u_pairs = take(sizeof(int4) * (size_t)np2), u_keys = take(4 * (size_t)np2),
                     u_perm = take(4 * (size_t)np2), u_sort = take(stable_sort_tmp_bytes(np2, (int32_t)nblk));
        const size_t tmp2_bytes = off;
        if (over_memory_limit(pool_bytes + tmp_bytes + pool2_bytes + tmp2_bytes))
            return fail_free(MBA_ERR_OOM, "device memory limit: the batch needs more");
        if (cudaMalloc(&b->pool2, pool2_bytes) != cudaSuccess || cudaMalloc(&tmp2, tmp2_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail_free(MBA_ERR_OOM, "device allocation of the batch failed");
        }
        char *b2 = (char *)b->pool2, *t2 = (char *)tmp2;
        A.pairs = (const int4 *)(b2 + o_pairs);
        A.Jcm = b2 + o_jcm;
        A.S = b2 + o_S;
        A.smax = smax;
        int4 *gen = (int4 *)(t2 + u_pairs);
        int32_t *keys = (int32_t *)(t2 + u_keys), *perm = (int32_t *)(t2 + u_perm);
        if (np2 > 0) {
            lay_pairs_kernel<<<lay_grid(NP), kLayBlock, 0, s>>>(NP, nw, po32, b->desc, pt_ptr, A.pm_pc, A.pm2cm,
                                                                nullptr, nullptr, pcnt, gen, keys, true);
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = stable_sort_by_key(keys, np2, (int32_t)nblk, perm, (int32_t *)A.blk_ptr, t2 + u_sort,
                                       stable_sort_tmp_bytes(np2, (int32_t)nblk), s);
            if (e == cudaSuccess) {
                lay_gather_pairs_kernel<<<lay_grid(np2), kLayBlock, 0, s>>>(np2, perm, gen, (int4 *)A.pairs);
                e = cudaGetLastError();
            }
        } else {
            e = cudaMemsetAsync((void *)A.blk_ptr, 0, 4 * ((size_t)nblk + 1), s);
        }
    }
    if (e == cudaSuccess) e = up(b->cams0, cameras, 72 * (size_t)NC);
    if (e == cudaSuccess) e = up(b->pts0, points, 24 * (size_t)NP);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.grad_obs, 0, 16 * (size_t)N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.grad_c0, 0, 72 * (size_t)NC, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.grad_p0, 0, 24 * (size_t)NP, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_free(MBA_ERR_CUDA, std::string("layout: ") + cudaGetErrorString(e));
    cudaFree(tmp);
    tmp = nullptr;
    if (tmp2) cudaFree(tmp2);
    tmp2 = nullptr;
    mba_status st = resolve_schedule(b, 0, 0, 0, &b->nt, &b->cps, &b->schur);
    if (st != MBA_OK) {
        std::string msg = mba_last_error();
        mba_batch_destroy(b);
        return api_fail(st, msg.c_str());
    }
    *out = b;
    return MBA_OK;
}

mba_status mba_batch_window_times(const mba_batch *b, double *ms) {
    if (!b || !ms) return api_fail(MBA_ERR_INVALID_ARG, "NULL argument");
    if (b->last_win_ns.size() != (size_t)b->nw) return api_fail(MBA_ERR_INVALID_ARG, "no solve yet");
    for (int w = 0; w < b->nw; ++w) ms[w] = 1e-6 * (double)b->last_win_ns[w];
    return MBA_OK;
}

void mba_batch_destroy(mba_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->pool) cudaFree(b->pool);
    if (b->pool2) cudaFree(b->pool2);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

mba_status mba_batch_info(const mba_batch *b, int32_t *n_windows, int64_t *n_cameras, int64_t *n_points,
                          int64_t *n_observations, int32_t *max_window_cameras) {
    if (!b) return api_fail(MBA_ERR_INVALID_ARG, "batch is NULL");
    if (n_windows) *n_windows = b->nw;
    if (n_cameras) *n_cameras = b->nc;
    if (n_points) *n_points = b->np;
    if (n_observations) *n_observations = b->n;
    if (max_window_cameras) *max_window_cameras = b->ncmax;
    return MBA_OK;
}

mba_status mba_batch_set_schedule(mba_batch *b, const mba_batch_schedule *sc) {
    if (!b || !sc) return api_fail(MBA_ERR_INVALID_ARG, "NULL argument");
    int nt = 0, cps = 0, schur = 0;
    mba_status st = resolve_schedule(b, sc->threads_per_cta, sc->ctas_per_sm, sc->schur, &nt, &cps, &schur);
    if (st != MBA_OK) return st;
    b->nt = nt;
    b->cps = cps;
    b->schur = schur;
    return MBA_OK;
}

mba_status mba_batch_get_schedule(const mba_batch *b, mba_batch_schedule *sc) {
    if (!b || !sc) return api_fail(MBA_ERR_INVALID_ARG, "NULL argument");
    sc->threads_per_cta = b->nt;
    sc->ctas_per_sm = b->cps;
    sc->schur = b->schur;
    return MBA_OK;
}

mba_status mba_batch_solve(mba_batch *b, const mba_solver_options *opt, const mba_batch_adjoint *adj,
                           mba_window_summary *summaries, double *ms) {
    if (!b) return api_fail(MBA_ERR_INVALID_ARG, "batch is NULL");
    mba_solver_options o;
    mba_solver_options_default(&o);
    if (opt) o = *opt;
    if (o.max_iter < 0 || o.pcg_max_iter < 0 || !(o.pcg_rel_tol >= 0.0) || !(o.initial_radius > 0.0) ||
        (o.damping != MBA_DAMP_DIAG && o.damping != MBA_DAMP_IDENTITY))
        return api_fail(MBA_ERR_INVALID_ARG, "bad solver options");
    if ((o.preconditioner != MBA_PRECOND_BLOCK_JACOBI && o.preconditioner != MBA_PRECOND_SCHUR_JACOBI) ||
        (o.forcing != 0 && o.forcing != 1) ||
        (o.pcg_variant != MBA_PCG_STANDARD && o.pcg_variant != MBA_PCG_SINGLE_REDUCTION))
        return api_fail(MBA_ERR_INVALID_ARG, "bad preconditioner, forcing or PCG variant option");
    if (o.preconditioner == MBA_PRECOND_SCHUR_JACOBI && !b->explicit_ok)
        return api_fail(MBA_ERR_INVALID_ARG, "the Schur-Jacobi preconditioner needs the explicit Schur form");
    if (adj && (!adj->grad_cameras || !adj->grad_points || adj->pcg_max_iter < 0 || !(adj->pcg_rel_tol >= 0.0)))
        return api_fail(MBA_ERR_INVALID_ARG, "bad adjoint arguments");
    cudaStream_t s = b->stream;
    BatchOpts bo{};
    bo.max_iter = o.max_iter;
    bo.pcg_max_iter = o.pcg_max_iter;
    bo.damping = o.damping;
    bo.adjoint = adj ? 1 : 0;
    bo.adj_pcg_max = adj ? adj->pcg_max_iter : 0;
    bo.pcg_tol = o.pcg_rel_tol;
    bo.initial_radius = o.initial_radius;
    bo.min_rel_dec = o.min_relative_decrease;
    bo.function_tol = o.function_tol;
    bo.adj_pcg_tol = adj ? adj->pcg_rel_tol : 0.0;
    bo.adj_mu = adj ? adj->mu : -1.0;
    // the Schur-Jacobi blocks come from the explicit S~, so that variant runs the explicit form
    bo.explicit_schur = (b->schur == 2 || o.preconditioner == MBA_PRECOND_SCHUR_JACOBI) ? 1 : 0;
    bo.precond = o.preconditioner;
    bo.forcing = o.forcing;
    bo.pcg_variant = o.pcg_variant;
    BCK(cudaMemcpyAsync(b->opts, &bo, sizeof(bo), cudaMemcpyHostToDevice, s));
    if (adj) {
        BCK(cudaMemcpyAsync(b->gbar_c, adj->grad_cameras, 72 * (size_t)b->nc, cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(b->gbar_p, adj->grad_points, 24 * (size_t)b->np, cudaMemcpyHostToDevice, s));
    }
    mba_status st = build_graph(b);
    if (st != MBA_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        BCK(cudaEventCreate(&e0));
        BCK(cudaEventCreate(&e1));
        BCK(cudaEventRecord(e0, s));
    }
    BCK(cudaGraphLaunch(b->gexec, s));
    if (ms) BCK(cudaEventRecord(e1, s));
    std::vector<mba_window_summary> sum((size_t)b->nw);
    BCK(cudaMemcpyAsync(sum.data(), b->out, sizeof(mba_window_summary) * b->nw, cudaMemcpyDeviceToHost, s));
    std::vector<unsigned long long> wns((size_t)b->nw);
    BCK(cudaMemcpyAsync(wns.data(), b->A.win_ns, 8 * (size_t)b->nw, cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    // The next launch claims the windows longest-first by this launch's measured
    // times (longest-processing-time-first on measured durations; the first
    // launch of a batch orders by observation count).  The order only decides
    // which CTA takes a window and when: every window's arithmetic, and so its
    // result, is the same in any order.
    {
        std::vector<int32_t> ord((size_t)b->nw);
        for (int w = 0; w < b->nw; ++w) ord[w] = w;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return wns[x] > wns[y]; });
        BCK(cudaMemcpyAsync(b->order, ord.data(), 4 * (size_t)b->nw, cudaMemcpyHostToDevice, s));
        BCK(cudaStreamSynchronize(s));
        b->last_win_ns.assign(wns.begin(), wns.end());
    }
    if (ms) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (adj) b->has_grads = true;
    if (summaries) std::memcpy(summaries, sum.data(), sizeof(mba_window_summary) * b->nw);
    for (int w = 0; w < b->nw; ++w)
        if (sum[w].status != MBA_OK) {
            char buf[96];
            std::snprintf(buf, sizeof(buf), "window %d: %s", w, mba_status_string((mba_status)sum[w].status));
            return api_fail((mba_status)sum[w].status, buf);
        }
    return MBA_OK;
}

mba_status mba_batch_autotune(mba_batch *b, const mba_solver_options *opt, mba_batch_schedule *chosen,
                              double *ms_best) {
    if (!b) return api_fail(MBA_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = b->stream;
    BCK(cudaMemcpyAsync(b->cams_bak, b->A.cams, 72 * (size_t)b->nc, cudaMemcpyDeviceToDevice, s));
    BCK(cudaMemcpyAsync(b->pts_bak, b->A.pts, 24 * (size_t)b->np, cudaMemcpyDeviceToDevice, s));
    const int nt0 = b->nt, cps0 = b->cps, sc0 = b->schur;
    double best = -1.0;
    int bnt = nt0, bcps = cps0, bsc = sc0;
    // one untimed solve first, so that every timed schedule claims the windows in
    // the order of measured times (and none pays the first launch's set-up)
    {
        mba_status st = mba_batch_solve(b, opt, nullptr, nullptr, nullptr);
        BCK(cudaMemcpyAsync(b->A.cams, b->cams_bak, 72 * (size_t)b->nc, cudaMemcpyDeviceToDevice, s));
        BCK(cudaMemcpyAsync(b->A.pts, b->pts_bak, 24 * (size_t)b->np, cudaMemcpyDeviceToDevice, s));
        BCK(cudaStreamSynchronize(s));
        if (st != MBA_OK && st != MBA_ERR_NONFINITE) return st;
    }
    const int nts[2] = {256, 512};
    for (int sch = b->explicit_ok ? 2 : 1; sch >= 1; --sch)
    for (int a = 0; a < 2; ++a) {
        for (int c = 1; c <= kMaxCtasPerSm; ++c) {
            if (max_ctas_per_sm(b, nts[a], c) < c) break;
            b->nt = nts[a];
            b->cps = c;
            b->schur = sch;
            double t = 0.0;
            mba_status st = mba_batch_solve(b, opt, nullptr, nullptr, &t);
            BCK(cudaMemcpyAsync(b->A.cams, b->cams_bak, 72 * (size_t)b->nc, cudaMemcpyDeviceToDevice, s));
            BCK(cudaMemcpyAsync(b->A.pts, b->pts_bak, 24 * (size_t)b->np, cudaMemcpyDeviceToDevice, s));
            BCK(cudaStreamSynchronize(s));
            if (st != MBA_OK && st != MBA_ERR_NONFINITE) {
                b->nt = nt0;
                b->cps = cps0;
                b->schur = sc0;
                return st;
            }
            if (best < 0.0 || t < best) {
                best = t;
                bnt = nts[a];
                bcps = c;
                bsc = sch;
            }
        }
    }
    b->nt = bnt;
    b->cps = bcps;
    b->schur = bsc;
    if (chosen) {
        chosen->threads_per_cta = bnt;
        chosen->ctas_per_sm = bcps;
        chosen->schur = bsc;
    }
    if (ms_best) *ms_best = best;
    return MBA_OK;
}

mba_status mba_batch_get_parameters(const mba_batch *b, double *cameras, double *points) {
    if (!b) return api_fail(MBA_ERR_INVALID_ARG, "batch is NULL");
    if (cameras) BCK(cudaMemcpyAsync(cameras, b->A.cams, 72 * (size_t)b->nc, cudaMemcpyDeviceToHost, b->stream));
    if (points) BCK(cudaMemcpyAsync(points, b->A.pts, 24 * (size_t)b->np, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return MBA_OK;
}

mba_status mba_batch_set_parameters(mba_batch *b, const double *cameras, const double *points) {
    if (!b) return api_fail(MBA_ERR_INVALID_ARG, "batch is NULL");
    if ((cameras && !finite_all(cameras, 9 * b->nc)) || (points && !finite_all(points, 3 * b->np)))
        return api_fail(MBA_ERR_NONFINITE, "non-finite parameters");
    if (cameras) BCK(cudaMemcpyAsync(b->A.cams, cameras, 72 * (size_t)b->nc, cudaMemcpyHostToDevice, b->stream));
    if (points) BCK(cudaMemcpyAsync(b->A.pts, points, 24 * (size_t)b->np, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return MBA_OK;
}

mba_status mba_batch_reset(mba_batch *b) {
    if (!b) return api_fail(MBA_ERR_INVALID_ARG, "batch is NULL");
    BCK(cudaMemcpyAsync(b->A.cams, b->cams0, 72 * (size_t)b->nc, cudaMemcpyDeviceToDevice, b->stream));
    BCK(cudaMemcpyAsync(b->A.pts, b->pts0, 24 * (size_t)b->np, cudaMemcpyDeviceToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return MBA_OK;
}

mba_status mba_batch_get_gradients(const mba_batch *b, double *grad_obs, double *grad_init_cam,
                                   double *grad_init_pt) {
    if (!b) return api_fail(MBA_ERR_INVALID_ARG, "batch is NULL");
    if (!b->has_grads) return api_fail(MBA_ERR_INVALID_ARG, "no solve with an adjoint has run");
    if (grad_obs) BCK(cudaMemcpyAsync(grad_obs, b->A.grad_obs, 16 * (size_t)b->n, cudaMemcpyDeviceToHost, b->stream));
    if (grad_init_cam)
        BCK(cudaMemcpyAsync(grad_init_cam, b->A.grad_c0, 72 * (size_t)b->nc, cudaMemcpyDeviceToHost, b->stream));
    if (grad_init_pt)
        BCK(cudaMemcpyAsync(grad_init_pt, b->A.grad_p0, 24 * (size_t)b->np, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return MBA_OK;
}

}  // extern "C"
