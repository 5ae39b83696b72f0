// mba_internal.cuh -- device data layout, camera model and shared device helpers
// of the GB300 bundle-adjustment library.  Everything here is internal to
// libmba.so; the public interface is include/mba.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>

#include "../../include/mba.h"
#include "edge_bal.cuh"

namespace mba {

constexpr int kBlock = 256;          // threads per CTA for every kernel
constexpr int kWarps = kBlock / 32;
constexpr int kCamTab = 28;          // values per camera in the camera table
constexpr int kVec = 12;             // padded stride of 9-vectors per camera (16-B aligned rows)
constexpr int kRow = 12;             // floats per camera row of the factored FP32 Schur product
// Staged point pass of the factored FP32 PCG: tiles of whole warp chunks copied
// into shared memory by 1-D bulk copies.  A tile holds at most kTileObs
// observations, kTilePts points and kTileChunks chunks; a stage holds one tile:
// per observation the camera index, the camera-major position of s, W Jp (6) and
// (px, py, 1/Pz) (3), each row with 8 words of slack for 16-byte rounding, then
// the points' C~^-1 (6 floats each), their CSR offsets and the chunk table.
constexpr int kTileObs = 1024, kTilePts = 384, kTileChunks = 31, kMaxStages = 4;
constexpr int kTileRow = kTileObs + 8;
constexpr int kStwSo = kTileRow, kStwJh = 2 * kTileRow, kStwPx = 8 * kTileRow, kStwCinv = 11 * kTileRow;
constexpr int kStwPtp = kStwCinv + 6 * kTilePts + 8, kStwWch = kStwPtp + kTilePts + 8;
constexpr int kStageWords = kStwWch + 2 * (kTileChunks + 4);
constexpr int kStageBytes = (kStageWords * 4 + 127) & ~127;
static_assert(kTileRow % 4 == 0 && kStwCinv % 4 == 0 && kStwPtp % 4 == 0 && kStwWch % 4 == 0,
              "16-byte aligned stage rows");
constexpr int kCamChunk = 256;       // observations per camera-major chunk (at least)
constexpr int kMaxTrack = 1024;      // longest supported point track

// Threads per CTA of the persistent PCG kernel (one CTA per SM): the FP32 form
// fits 64 registers per thread, the FP64 form needs up to 128.
template <typename T>
struct PcgBlock {
    static constexpr int value = sizeof(T) == 4 ? 1024 : 512;
};

// Device-resident LM / PCG control state.  All LM decisions are made on the
// device so a whole solve is issued without host round trips.
struct DevState {
    double radius, factor, mu;
    double cost;          // F(x) at the current parameters
    double initial_cost;
    double cost_new, model_dec, gain;
    double pcg_rel_res;
    double mu_override;   // >= 0: use this mu instead of 1/radius
    double mu_accepted;   // mu of the last accepted step (the step that produced the current x)
    double g0;            // norm of the first reduced right-hand side of the solve (forcing sequence)
    int32_t relin;        // 1: the linearisation must be rebuilt before the next solve
    int32_t accepted;     // decision of the last iteration
    int32_t done;         // 1: stop issuing work (function_tol met or error)
    int32_t iter;
    int32_t err;          // mba_status raised on the device
    int32_t pcg_iters;
    int32_t accepted_total, pcg_total;
    uint32_t barrier;     // arrival counter of the persistent kernel's grid barrier
    int32_t blockfail;    // 1: a damped block was not positive definite in this iteration
};

// Everything a kernel needs, as plain device pointers.  Sized at creation.
struct Prob {
    int32_t nc, np;
    int64_t n, npad;       // observations, padded stride of SoA arrays
    int32_t fp32;          // 1: FP32-mixed
    int32_t loss;
    double delta;
    int32_t n_cchunks;
    // warp chunks: wchunk[w] = (first point, first observation); runs of whole
    // points with <= 32 observations, or a single point with a longer track
    int32_t n_wchunks;
    int2 *wchunk;          // n_wchunks + 1
    int32_t pcg_use_ps;    // 1: the search direction is copied into shared memory per pass
    int32_t pcg_smem;      // dynamic shared memory of the PCG kernel

    // parameters (FP64, row-major)
    double *cams, *pts;            // current
    double *cams_new, *pts_new;    // candidate
    double *cams0, *pts0;          // as given at creation

    // observations, point-major order (stable by point, then input index)
    int32_t *pm_cam, *pm_pt, *pm_orig;
    double2 *pm_uv;
    int32_t *pt_ptr;               // np + 1
    // observations, camera-major order
    int32_t *cm_pt, *cm_orig;
    double2 *cm_uv;
    int32_t *cam_ptr;              // nc + 1
    int32_t *pm2cm;                // per point-major position: its camera-major position
    // FP32-mixed: float copies of the pixels (point-major and camera-major, made at
    // creation) and of the current points (refreshed at every linearisation), so
    // the FP32 kernels convert nothing per observation (on GB300 a conversion from
    // FP64 runs on the FP64 pipe); null in FP64 problems
    float2 *pm_uv32, *cm_uv32;
    float4 *pts32;
    // nodes held constant (mba_set_fixed): nonzero bytes mark fixed cameras and
    // points; has_fixed = 0 while none is fixed, so no kernel reads the masks
    uint8_t *cam_fixed, *pt_fixed;
    int32_t has_fixed;
    // staged point pass (factored FP32 form): tiles (first chunk, end chunk) of
    // whole warp chunks with <= 32 observations, tile t worked by CTA t mod grid;
    // chunks of longer tracks are listed apart and read from global memory
    int2 *tiles;
    int4 *tdesc;            // per tile: (oa, ob, ca, cz), (pa, pz, wa, wz), (first chunk, end chunk, 0, 0):
                            // the 16-byte-rounded copy ranges of its observation rows, C~^-1 floats,
                            // CSR offsets and chunk entries
    int32_t n_tiles;
    int32_t *long_chunks;
    int32_t n_long;
    int32_t pcg_stages;     // stages of the staged point pass (0: not staged)
    int32_t pcg_stage_off;  // byte offset of the stages in the PCG kernel's dynamic shared memory
    // chunk tables
    int32_t *cchunk_cam, *cchunk_beg;  // n_cchunks, n_cchunks + 1
    int32_t *cfirst;               // nc + 1: first camera chunk of each camera
    int32_t *cta_cam;              // grid + 1: cameras owned by each PCG CTA (balanced by observations)
    int32_t pcg_max_cta_chunks;    // most camera chunks any PCG CTA owns
    int32_t pcg_ps_bytes;          // shared-memory bytes of the search-direction copy

    // per-linearisation data (T = float in FP32-mixed, double otherwise)
    void *J;        // [24][npad] sqrt(W)-scaled Jacobian, point-major (null in the factored form)
    void *res;      // [2][npad]  sqrt(W)-scaled residual
    void *camtab;   // [nc][kCamTab] camera table in T (lin kernels)
    double *camtab64;  // [nc][kCamTab] FP64 camera table (cost evaluation)
    double *Hpp;    // [nc][45] packed upper triangle of B
    double *v;      // [nc][9]
    double *Hll;    // [np][6] packed upper triangle of C
    double *w;      // [np][3]
    double *cpart;  // [n_cchunks][54] camera-chunk partial sums (the PCG reuses [n_cchunks][9])
    void *zT;       // FP32-mixed: [nc][kVec] float copy of z
    void *pT2;      // FP32-mixed: second float search-direction buffer (alternate iterations)
    double *Jcm;    // FP64: [18][npad] sqrt(W)-scaled camera Jacobian, camera-major
    // FP32-mixed analytic (factored) form: per observation the normalised point
    // and 1 / P_z (point-major), the point rotated into the camera frame, R X,
    // with 1 / P_z (camera-major), and the W-scaled point Jacobian, from which
    // the PCG re-derives Jc p and Jc^T s with per-camera constants
    float *PXpm;    // [3][npad] (px, py, 1/Pz), point-major
    float *Jph;     // [6][npad] W Jp, point-major
    float *RXcm;    // [npad] float4 (R X, 1/Pz), camera-major
    float *swpm;    // [npad] sqrt(W), point-major (factored form with a robust loss; else null)
    // float-float copies for the FP32-mixed solve's cost (ff.cuh; else null)
    float2 *camff;  // [nc][16] R (9), t (3), f, k1, k2 of the cost's camera table
    float4 *uvff;   // [n] observations, point-major (u hi, u lo, v hi, v lo)
    float2 *ptsff;  // [np][3] the points being evaluated
    int32_t fact;   // 1: the PCG runs the factored form (FP32-mixed, analytic Jacobian)
    void *JcmT;     // [18][npad] sqrt(W)-scaled camera Jacobian in T, camera-major, that the PCG
                    // camera pass reads: Jcm in FP64; FP32-mixed with autodiff only (else null)
    int32_t autodiff;  // 1: every Jacobian comes from the edge functor on dual numbers
    // per-solve data
    double *Bd;     // [nc][81] damped B~
    double *Binv;   // [nc][81] inverse of B~ (block-Jacobi preconditioner)
    void *Cinv;     // [np][6] packed inverse of damped C~, T
    // PCG vectors, [nc][kVec] FP64
    double *x, *r, *z, *p, *p2, *q, *g;  // p, p2: search directions of alternate iterations
    void *pT;       // [nc][kVec] search direction in T (point pass gathers when not in shared memory)
    void *sbuf;     // [npad] per observation s = Jp~ b (2 x T) in camera-major order, scattered by the point pass
    double *dp;     // [np][3] point step
    double *red;    // reduction partials: per-CTA p.q, r.z and r.r of the persistent kernel
    int32_t red_len;
    DevState *st;
    mba_iteration *trace;  // device trace, max_iter entries (set per solve)
    int32_t trace_cap;
};

// ---------------------------------------------------------------------------
// packed symmetric indexing
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int sym9(int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    return a * 9 - (a * (a - 1)) / 2 + (b - a);
}
__host__ __device__ __forceinline__ int sym3(int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    return a * 3 - (a * (a - 1)) / 2 + (b - a);
}

// ---------------------------------------------------------------------------
// BAL camera model.  Per camera (once per linearisation) the rotation R(w) and
// the factor M of dP/dw = -R [X]_x M, M = (w w^T + (R^T - I)[w]_x) / |w|^2
// (Gallego & Yezzi 2015) are tabulated in FP64; for |w|^2 <= DBL_EPSILON the
// first-order form P = X + w x X + t is used (R = I + [w]_x, dP/dw = -[X]_x).
// Table row: R[9] M[9] t[3] f k1 k2 small w[3] (w: the raw angle-axis, read by
// the dual-number path, which evaluates the edge functor from the parameters).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void camera_table_row(const double *c, double *o) {
    const double w0 = c[0], w1 = c[1], w2 = c[2];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double R[9], M[9];
    double small;
    if (th2 > DBL_EPSILON) {
        const double th = sqrt(th2);
        double s, co;
        sincos(th, &s, &co);
        const double k0 = w0 / th, k1 = w1 / th, k2 = w2 / th;
        const double oc = 1.0 - co;
        R[0] = co + oc * k0 * k0;      R[1] = -s * k2 + oc * k0 * k1; R[2] = s * k1 + oc * k0 * k2;
        R[3] = s * k2 + oc * k1 * k0;  R[4] = co + oc * k1 * k1;      R[5] = -s * k0 + oc * k1 * k2;
        R[6] = -s * k1 + oc * k2 * k0; R[7] = s * k0 + oc * k2 * k1;  R[8] = co + oc * k2 * k2;
        // (R^T - I) [w]_x, then add w w^T and divide by th^2
        const double A[9] = {R[0] - 1.0, R[3], R[6], R[1], R[4] - 1.0, R[7], R[2], R[5], R[8] - 1.0};
        const double W[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
        const double wv[3] = {w0, w1, w2};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                double acc = A[i * 3 + 0] * W[0 * 3 + j] + A[i * 3 + 1] * W[1 * 3 + j] + A[i * 3 + 2] * W[2 * 3 + j];
                M[i * 3 + j] = (acc + wv[i] * wv[j]) / th2;
            }
        small = 0.0;
    } else {
        R[0] = 1.0; R[1] = -w2; R[2] = w1;
        R[3] = w2;  R[4] = 1.0; R[5] = -w0;
        R[6] = -w1; R[7] = w0;  R[8] = 1.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) M[i] = (i % 4 == 0) ? 1.0 : 0.0;
        small = 1.0;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) { o[i] = R[i]; o[9 + i] = M[i]; }
    o[18] = c[3]; o[19] = c[4]; o[20] = c[5];
    o[21] = c[6]; o[22] = c[7]; o[23] = c[8];
    o[24] = small; o[25] = w0; o[26] = w1; o[27] = w2;
}

// Correctly rounded reciprocal (the same value as 1 / x, without the divide routine).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// Residual e = pi(c, X) - u and, if JAC, the analytic Jacobians Jc (2x9, row
// major: w, t, f, k1, k2) and Jp (2x3) by the chain rule, in precision T.
// pz (optional): the normalised point p = (px, py) and 1 / P_z.
template <typename T, bool JAC>
__device__ __forceinline__ void project(const T *__restrict__ ct, T X0, T X1, T X2, T u0, T u1, T *e, T *Jc,
                                        T *Jp, T *pz = nullptr) {
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
    e[0] = f * d * px - u0;
    e[1] = f * d * py - u1;
    if (pz) {
        pz[0] = px;
        pz[1] = py;
        pz[2] = iz;
    }
    if (!JAC) return;
    const T dd = T(2) * k1 + T(4) * k2 * r2;
    // A = d(pixel)/dp = f (d I + dd p p^T); D = A dp/dP
    const T a00 = f * (d + dd * px * px), a01 = f * dd * px * py, a11 = f * (d + dd * py * py);
    T D[6];
    D[0] = -a00 * iz; D[1] = -a01 * iz; D[2] = -(a00 * px + a01 * py) * iz;
    D[3] = -a01 * iz; D[4] = -a11 * iz; D[5] = -(a01 * px + a11 * py) * iz;
    // Jp = D R
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        Jp[r * 3 + 0] = D[r * 3] * R0 + D[r * 3 + 1] * R3 + D[r * 3 + 2] * R6;
        Jp[r * 3 + 1] = D[r * 3] * R1 + D[r * 3 + 1] * R4 + D[r * 3 + 2] * R7;
        Jp[r * 3 + 2] = D[r * 3] * R2 + D[r * 3 + 1] * R5 + D[r * 3 + 2] * R8;
    }
    const bool small = ct[24] != T(0);
    // rotation block: row r = (X x b_r)^T M with b = D R (or D in the first-order branch)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const T b0 = small ? D[r * 3] : Jp[r * 3];
        const T b1 = small ? D[r * 3 + 1] : Jp[r * 3 + 1];
        const T b2 = small ? D[r * 3 + 2] : Jp[r * 3 + 2];
        const T v0 = X1 * b2 - X2 * b1, v1 = X2 * b0 - X0 * b2, v2 = X0 * b1 - X1 * b0;
        Jc[r * 9 + 0] = v0 * ct[9] + v1 * ct[12] + v2 * ct[15];
        Jc[r * 9 + 1] = v0 * ct[10] + v1 * ct[13] + v2 * ct[16];
        Jc[r * 9 + 2] = v0 * ct[11] + v1 * ct[14] + v2 * ct[17];
        Jc[r * 9 + 3] = D[r * 3];
        Jc[r * 9 + 4] = D[r * 3 + 1];
        Jc[r * 9 + 5] = D[r * 3 + 2];
        const T pr = r == 0 ? px : py;
        Jc[r * 9 + 6] = d * pr;
        Jc[r * 9 + 7] = f * r2 * pr;
        Jc[r * 9 + 8] = f * r2 * r2 * pr;
    }
}

// The point and the pixels of an observation in the precision T of the
// linearisation: FP64 problems read the FP64 arrays, FP32-mixed problems their
// float copies (the same bits as converting here).
template <typename T>
__device__ __forceinline__ void load_point(const Prob &P, int pt, T &X0, T &X1, T &X2) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(P.pts32 + pt);
        X0 = v.x;
        X1 = v.y;
        X2 = v.z;
    } else {
        X0 = __ldg(P.pts + 3 * (int64_t)pt);
        X1 = __ldg(P.pts + 3 * (int64_t)pt + 1);
        X2 = __ldg(P.pts + 3 * (int64_t)pt + 2);
    }
}
template <typename T>
__device__ __forceinline__ void load_uv(const double2 *uv64, const float2 *uv32, int64_t o, T &u0, T &u1) {
    if constexpr (sizeof(T) == 4) {
        const float2 v = __ldg(uv32 + o);
        u0 = v.x;
        u1 = v.y;
    } else {
        const double2 v = __ldg(uv64 + o);
        u0 = v.x;
        u1 = v.y;
    }
}

// Nodes held constant (mba_set_fixed) have zero Jacobian columns, the convention
// of g2o / Ceres for fixed vertices that the paper's graph API follows (Sec.
// 5.3): their blocks, gradients and Schur couplings vanish, so their step is
// exactly zero and they stay bit-identical.  Jc or Jp may be null.
template <typename T>
__device__ __forceinline__ void zero_fixed_columns(const Prob &P, int cam, int pt, T *Jc, T *Jp) {
    if (!P.has_fixed) return;
    if (Jc && P.cam_fixed[cam]) {
#pragma unroll
        for (int q = 0; q < 18; ++q) Jc[q] = T(0);
    }
    if (Jp && P.pt_fixed[pt]) {
#pragma unroll
        for (int q = 0; q < 6; ++q) Jp[q] = T(0);
    }
}

// Residual and Jacobians of one observation from either source: the analytic
// chain rule (project) or the edge functor on dual numbers (AD), whose camera
// parameters come from the table row (w at 25..27, t, f, k1, k2 at 18..23).
// CAM / PT select the Jacobian blocks the dual-number path forms (kJetK
// directions per pass); the analytic path forms both.
constexpr int kJetK = 12;
template <typename T, bool AD, bool CAM = true, bool PT = true>
__device__ __forceinline__ void edge_eval(const T *__restrict__ ct, T X0, T X1, T X2, T u0, T u1, T *e, T *Jc,
                                          T *Jp, T *pz = nullptr) {
    if (!AD) {
        project<T, true>(ct, X0, X1, X2, u0, u1, e, Jc, Jp, pz);
        return;
    }
    const T cam[9] = {ct[25], ct[26], ct[27], ct[18], ct[19], ct[20], ct[21], ct[22], ct[23]};
    const T X[3] = {X0, X1, X2};
    T pix[2];
    jet_jacobian<(CAM && PT) ? kJetK : (CAM ? 9 : 3), CAM, PT>(Edge{}, cam, X, pix, Jc, Jp);
    e[0] = pix[0] - u0;
    e[1] = pix[1] - u1;
}
// Residual only.
template <typename T, bool AD>
__device__ __forceinline__ void edge_residual(const T *__restrict__ ct, T X0, T X1, T X2, T u0, T u1, T *e) {
    if (!AD) {
        project<T, false>(ct, X0, X1, X2, u0, u1, e, nullptr, nullptr);
        return;
    }
    const T cam[9] = {ct[25], ct[26], ct[27], ct[18], ct[19], ct[20], ct[21], ct[22], ct[23]};
    const T X[3] = {X0, X1, X2};
    T pix[2];
    Edge{}(cam, X, pix);
    e[0] = pix[0] - u0;
    e[1] = pix[1] - u1;
}

// Loss: rho(s) and IRLS weight rho'(s).  Plain: s, 1.  Huber: s, 1 for
// s <= delta^2, else 2 delta sqrt(s) - delta^2, delta / sqrt(s).
template <typename T>
__device__ __forceinline__ void loss_weight(int loss, T delta, T s, T *rho, T *weight) {
    if (loss == MBA_LOSS_HUBER && s > delta * delta) {
        const T r = sqrt(s);
        *rho = T(2) * delta * r - delta * delta;
        *weight = delta / r;
    } else {
        *rho = s;
        *weight = T(1);
    }
}

// ---------------------------------------------------------------------------
// L2-coherent loads/stores for data that other CTAs write inside the same
// persistent launch (L1 is not coherent across SMs).
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void stcg(T *p, T v) { __stcg(p, v); }

// Block-wide sum of one double per thread in a fixed tree order (shuffles in
// each warp, then across the warp sums in warp 0); result valid in thread 0.
// sbuf holds one double per warp (up to 32).
__device__ __forceinline__ double block_sum(double v, double *sbuf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sbuf[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < (int)(blockDim.x >> 5) ? sbuf[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// Bounded grid barrier for cooperative (co-resident) launches.  Arrivals
// increment a monotone counter (release); the k-th barrier completes when an
// acquire load sees k * gridDim.x.  A CTA that polls more than `limit` times, or sees the error
// flag raised, records MBA_ERR_TIMEOUT and returns false; the caller must
// then leave the kernel.  Returns true when every CTA has arrived.
// ---------------------------------------------------------------------------
// mbarrier and 1-D bulk copy (cp.async.bulk) helpers for shared-memory staging.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// one arrival that also expects `bytes` of bulk-copy completions in this phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// wait for the phase of the given parity to complete; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) completing on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool grid_barrier(DevState *st, uint32_t &epoch, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        const uint32_t target = epoch * gridDim.x;
        unsigned int *ctr = reinterpret_cast<unsigned int *>(&st->barrier);
        // release: the CTA's writes (ordered before this thread by the block
        // barrier above) become visible to every CTA whose acquire load below
        // sees this arrival
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(ctr), "r"(1u) : "memory");
        int ok = 1;
        long long polls = 0;
        for (;;) {
            unsigned int seen;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(ctr) : "memory");
            if ((int)(seen - target) >= 0) break;
            int e;
            asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(e) : "l"(&st->err) : "memory");
            if (e != 0 || ++polls > limit) {
                atomicCAS(&st->err, 0, (int)MBA_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(16);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// host launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// sort.cu
cudaError_t stable_sort_by_key(const int32_t *keys_in, int64_t n, int32_t nkeys, int32_t *perm_out,
                               int32_t *ptr_out, void *tmp, size_t tmp_bytes, cudaStream_t s);
size_t stable_sort_tmp_bytes(int64_t n, int32_t nkeys);
int64_t exclusive_scan_tmp_ints(int64_t n);
cudaError_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s);
cudaError_t validate_inputs(const double *cams, int32_t nc, const double *pts, int32_t np, const double *obs,
                            const int32_t *ci, const int32_t *pi, int64_t n, int32_t *flags, cudaStream_t s);
cudaError_t gather_layout(Prob &P, const double *obs_in, const int32_t *ci, const int32_t *pi, int32_t *max_track,
                          int32_t *tmp_i, cudaStream_t s);
cudaError_t build_pm2cm(Prob &P, int32_t *tmp_n, cudaStream_t s);

// linearize.cu
cudaError_t launch_camera_tables(const Prob &P, const double *cams, bool for_lin, cudaStream_t s);
cudaError_t launch_camera_tables_forced(const Prob &P, const double *cams, cudaStream_t s);
cudaError_t launch_linearize_impl(const Prob &P, const int32_t *cfirst, int force, cudaStream_t s);
// ff: evaluate in float-float arithmetic (FP32-mixed solves; ff.cuh)
cudaError_t launch_cost_impl(const Prob &P, const double *pts, double *partial, double *out, double *out2, int gate,
                             cudaStream_t s, bool ff = false);
cudaError_t launch_split_observations(const Prob &P, cudaStream_t s);
int cost_grid(const Prob &P);
cudaError_t launch_evaluate_slice(const Prob &P, const int32_t *ci, const int32_t *pi, const double2 *uv, int64_t m,
                                  double *e, double *jc, double *jp, cudaStream_t s);

// pcg.cu
enum PcgMode { PCG_SOLVE = 0, PCG_RHS_ONLY = 1, PCG_MATVEC = 2 };
cudaError_t launch_damp(const Prob &P, int damping, int precond, const int32_t *cfirst, cudaStream_t s);
// variant: mba_pcg_variant (STANDARD: Alg. 2; SINGLE_REDUCTION: the Chronopoulos-Gear form)
cudaError_t launch_pcg(const Prob &P, int mode, int max_iter, double tol, long long spin_limit, int grid,
                       cudaStream_t s, int forcing = 0, int variant = 0);
int pcg_grid_size(const Prob &P);
void plan_pcg_smem(Prob &P);
cudaError_t launch_backsub(const Prob &P, double *partial, int nb, cudaStream_t s);

// adjoint.cu
cudaError_t launch_adjoint_obs(const Prob &P, const int32_t *ci, const int32_t *pi, const double2 *uv, int64_t m,
                               double *out, cudaStream_t s);
cudaError_t launch_adjoint_init(const Prob &P, int damping, double mu, cudaStream_t s);

// api.cu: records msg as the calling thread's mba_last_error() text and returns st
mba_status api_fail(mba_status st, const char *msg);
// true if a creation needing `bytes` of device memory exceeds the cap set by
// mba_set_device_memory_limit
bool over_memory_limit(size_t bytes);

// lm.cu
cudaError_t launch_state_init(const Prob &P, double radius, double mu_override, int keep_cost, cudaStream_t s);
cudaError_t launch_lm_update(const Prob &P, const mba_solver_options &o, cudaStream_t s);
cudaError_t launch_accept(const Prob &P, cudaStream_t s);

}  // namespace mba
