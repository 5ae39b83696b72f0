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
// preconditioner; C~^-1 (adjugate, FP64) is stored packed in T.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double damp_term(int damping, double d) {
    if (damping == MBA_DAMP_IDENTITY) return 1.0;
    return fmin(fmax(d, 1e-6), 1e32);
}

__device__ __forceinline__ double current_mu(const DevState *st) {
    return st->mu_override >= 0.0 ? st->mu_override : 1.0 / st->radius;
}

__global__ void damp_cameras_kernel(Prob P, int damping) {
    DevState *st = P.st;
    if (st->done) return;
    const double mu = current_mu(st);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->mu = mu;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.nc; i += gridDim.x * blockDim.x) {
        double A[81];
#pragma unroll
        for (int a = 0; a < 9; ++a)
#pragma unroll
            for (int b = 0; b < 9; ++b) A[a * 9 + b] = P.Hpp[45 * (int64_t)i + sym9(a, b)];
#pragma unroll
        for (int a = 0; a < 9; ++a) A[a * 10] += mu * damp_term(damping, A[a * 10]);
        for (int q = 0; q < 81; ++q) P.Bd[81 * (int64_t)i + q] = A[q];
        // lower Cholesky in place
        bool ok = true;
        for (int j = 0; j < 9; ++j) {
            double s = A[j * 9 + j];
            for (int k = 0; k < j; ++k) s -= A[j * 9 + k] * A[j * 9 + k];
            if (!(s > 0.0)) { ok = false; break; }
            const double l = sqrt(s);
            A[j * 9 + j] = l;
            for (int r = j + 1; r < 9; ++r) {
                double t = A[r * 9 + j];
                for (int k = 0; k < j; ++k) t -= A[r * 9 + k] * A[j * 9 + k];
                A[r * 9 + j] = t / l;
            }
        }
        if (!ok) {
            atomicCAS(&st->err, 0, (int)MBA_ERR_NONFINITE);
            continue;
        }
        // inverse = L^-T L^-1, column by column
        for (int col = 0; col < 9; ++col) {
            double y[9];
            for (int r = 0; r < 9; ++r) {
                double s = (r == col) ? 1.0 : 0.0;
                for (int k = 0; k < r; ++k) s -= A[r * 9 + k] * y[k];
                y[r] = s / A[r * 9 + r];
            }
            for (int r = 8; r >= 0; --r) {
                double s = y[r];
                for (int k = r + 1; k < 9; ++k) s -= A[k * 9 + r] * y[k];
                y[r] = s / A[r * 9 + r];
            }
            for (int r = 0; r < 9; ++r) P.Binv[81 * (int64_t)i + r * 9 + col] = y[r];
        }
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
            atomicCAS(&st->err, 0, (int)MBA_ERR_NONFINITE);
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
// shared pieces of the point-major passes
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void load_jac(const T *__restrict__ J, int64_t npad, int64_t o, T *Jc, T *Jp) {
#pragma unroll
    for (int q = 0; q < 18; ++q) Jc[q] = __ldg(J + q * npad + o);
#pragma unroll
    for (int q = 0; q < 6; ++q) Jp[q] = __ldg(J + (18 + q) * npad + o);
}

__device__ __forceinline__ void acc_camera(float *row, const float *y) {
    atomicAdd(reinterpret_cast<float4 *>(row), make_float4(y[0], y[1], y[2], y[3]));
    atomicAdd(reinterpret_cast<float4 *>(row + 4), make_float4(y[4], y[5], y[6], y[7]));
    atomicAdd(row + 8, y[8]);
}
__device__ __forceinline__ void acc_camera(double *row, const double *y) {
#pragma unroll
    for (int q = 0; q < 9; ++q) atomicAdd(row + q, y[q]);
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
// Warp-granular point pass.  The point-major observation stream is cut, at
// creation, into warp chunks: runs of whole points with at most 32
// observations (one lane per observation), or one point with a longer track
// on its own.  A warp owns its chunks outright, so the per-point sums need
// only shuffles (a segmented scan keyed by point) and no block barriers; other
// warps on the SM hide each chunk's load latency.
// ---------------------------------------------------------------------------
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

// E b contribution of one observation, added into its camera: y = Jc^T (Jp b)
template <typename T>
__device__ __forceinline__ void e_b(const T *Jc, const T *Jp, const T *b, T *acc_row) {
    const T s0 = Jp[0] * b[0] + Jp[1] * b[1] + Jp[2] * b[2];
    const T s1 = Jp[3] * b[0] + Jp[4] * b[1] + Jp[5] * b[2];
    T y[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) y[a] = Jc[a] * s0 + Jc[9 + a] * s1;
    acc_camera(acc_row, y);
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

// One pass of the implicit Schur product over the warp chunks of this CTA.
// RHS: b_j = C~_j^-1 w_j.  Otherwise b_j = C~_j^-1 sum_k Jp~_k^T Jc~_k p_i(k).
// Then Jc~_k^T Jp~_k b_j is added into acc[i(k)].  Per chunk the dependent
// loads are: (point, camera) of each lane, then Jacobian, C~^-1 of the lane's
// point and the camera's p together; the next chunk's table entries are
// fetched one chunk ahead.
template <typename T, bool RHS>
__device__ void point_pass(const Prob &P, const T *ps, const T *pT, T *acc) {
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
            const int2 pc = act ? P.pm_pc[o] : make_int2(-1 - lane, 0);
            const int pt = pc.x, cam = pc.y;
            T Jc[18], Jp[6], ci[6];
            if (act) {
                load_jac(J, npad, o, Jc, Jp);
                load_sym3(Cinv + 6 * (int64_t)pt, ci);
            } else {
#pragma unroll
                for (int q = 0; q < 18; ++q) Jc[q] = T(0);
#pragma unroll
                for (int q = 0; q < 6; ++q) Jp[q] = ci[q] = T(0);
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
                // inclusive segmented scan keyed by point (segments are contiguous)
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
            if (act) e_b(Jc, Jp, b, acc + (int64_t)cam * kVec);
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
                        load_jac(J, npad, o, Jc, Jp);
                        gather_p(ps, pT, P.pm_pc[o].y, pa);
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
                    T Jc[18], Jp[6];
                    load_jac(J, npad, o, Jc, Jp);
                    e_b(Jc, Jp, b, acc + (int64_t)P.pm_pc[o].y * kVec);
                }
            }
        }
        c0 = n0;
        c1 = n1;
    }
}

// Copy the search direction into shared memory (dense nc x 9).
template <typename T>
__device__ void stage_p(const Prob &P, const T *pT, T *ps) {
    const int total = P.nc * 9;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int cam = e / 9, a = e - cam * 9;
        ps[e] = ldcg(pT + (int64_t)cam * kVec + a);
    }
    __syncthreads();
}

// Sum of the per-CTA partials in a fixed order (every CTA gets the same value).
__device__ __forceinline__ double sum_parts(const double *parts, int G, double *sb) {
    __shared__ double s_out;
    double acc = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) acc += ldcg(parts + i);
    const double s = block_sum(acc, sb);
    if (threadIdx.x == 0) s_out = s;
    __syncthreads();
    return s_out;
}

// ---------------------------------------------------------------------------
// persistent PCG kernel (cooperative launch, one CTA set for the whole solve)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kPcgBlock, sizeof(T) == 4 ? 4 : 2) pcg_kernel(Prob P, int mode, int max_iter, double tol, long long spin) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double sb[32];
    DevState *st = P.st;
    if (st->done) return;
    uint32_t epoch = 0;
    const int G = gridDim.x;
    const int nwarp = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t vec_n = (int64_t)P.nc * kVec;
    T *pT = (T *)P.pT;
    T *cacc0 = (T *)P.cacc, *cacc1 = cacc0 + vec_n;
    double *part_pq = P.red, *part_rho = P.red + G, *part_rr = P.red + 2 * G;
    const int ncw = (P.nc + 2) / 3;  // warps of camera work (3 cameras x 9 rows per warp)
    const int my_sub = lane / 9, row = lane % 9;
    const unsigned full = 0xffffffffu;

    T *ps = P.pcg_use_ps ? (T *)smem_raw : nullptr;
    bool ok = true;
    auto barrier = [&]() -> bool { return grid_barrier(st, epoch, spin); };

    if (mode == PCG_MATVEC) {
        // p given in P.p (FP64): q = B~ p - E C~^-1 E^T p
        for (int w = blockIdx.x * nwarp + wid; w < ncw; w += G * nwarp) {
            const int cam = w * 3 + my_sub;
            if (lane < 27 && cam < P.nc) stcg(pT + (int64_t)cam * kVec + row, (T)P.p[(int64_t)cam * kVec + row]);
        }
        ok = barrier();
        if (ok && ps) stage_p(P, pT, ps);
        if (ok) point_pass<T, false>(P, ps, pT, cacc0);
        if (ok) ok = barrier();
        if (ok) {
            for (int w = blockIdx.x * nwarp + wid; w < ncw; w += G * nwarp) {
                const int cam = w * 3 + my_sub;
                const bool act = lane < 27 && cam < P.nc;
                const int64_t vo = (int64_t)(act ? cam : 0) * kVec;
                const double pr = act ? P.p[vo + row] : 0.0;
                double bp = 0.0;
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    const double pc = __shfl_sync(full, pr, my_sub * 9 + c);
                    if (act) bp += P.Bd[81 * (int64_t)cam + row * 9 + c] * pc;
                }
                if (act) P.q[vo + row] = bp - (double)ldcg(cacc0 + vo + row);
            }
        }
        return;
    }

    // ---- right-hand side g = v - E C~^-1 w (Eq. 3) into cacc1 ----
    point_pass<T, true>(P, nullptr, pT, cacc1);
    ok = barrier();
    if (ok) {
        double rr = 0.0, rz = 0.0;
        for (int w = blockIdx.x * nwarp + wid; w < ncw; w += G * nwarp) {
            const int cam = w * 3 + my_sub;
            const bool act = lane < 27 && cam < P.nc;
            const int64_t vo = (int64_t)(act ? cam : 0) * kVec;
            double g = 0.0;
            if (act) {
                g = P.v[9 * (int64_t)cam + row] - (double)ldcg(cacc1 + vo + row);
                P.g[vo + row] = g;
                P.x[vo + row] = 0.0;
                P.r[vo + row] = g;
            }
            double z = 0.0;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                const double gc = __shfl_sync(full, g, my_sub * 9 + c);
                if (act) z += P.Binv[81 * (int64_t)cam + row * 9 + c] * gc;
            }
            if (act) {
                P.z[vo + row] = z;
                rr += g * g;
                rz += g * z;
            }
        }
        if (mode == PCG_RHS_ONLY) return;
        const double s_rr = block_sum(rr, sb);
        const double s_rz = block_sum(rz, sb);
        if (threadIdx.x == 0) {
            stcg(part_rr + blockIdx.x, s_rr);
            stcg(part_rho + blockIdx.x, s_rz);
        }
        ok = barrier();
    }

    int n = 0;
    double r0 = 0.0, rho_prev = 0.0, rn = 0.0;
    if (ok) {
        r0 = sqrt(sum_parts(part_rr, G, sb));
        rn = r0;
    }
    if (ok && r0 > 0.0) {
        for (;;) {
            const double rho = sum_parts(part_rho, G, sb);
            if (!isfinite(rho)) break;
            const double beta = n == 0 ? 0.0 : rho / rho_prev;
            // phase P: p = z + beta p
            for (int w = blockIdx.x * nwarp + wid; w < ncw; w += G * nwarp) {
                const int cam = w * 3 + my_sub;
                if (lane < 27 && cam < P.nc) {
                    const int64_t vo = (int64_t)cam * kVec + row;
                    const double pn = n == 0 ? P.z[vo] : fma(beta, P.p[vo], P.z[vo]);
                    P.p[vo] = pn;
                    stcg(pT + vo, (T)pn);
                }
            }
            if (!(ok = barrier())) break;
            // phase A: E C~^-1 E^T p
            T *acc = (n & 1) ? cacc1 : cacc0;
            T *acc_next = (n & 1) ? cacc0 : cacc1;
            if (ps) stage_p(P, pT, ps);
            point_pass<T, false>(P, ps, pT, acc);
            if (!(ok = barrier())) break;
            // phase Q: q = B~ p - acc; p.q
            {
                double pq = 0.0;
                for (int w = blockIdx.x * nwarp + wid; w < ncw; w += G * nwarp) {
                    const int cam = w * 3 + my_sub;
                    const bool act = lane < 27 && cam < P.nc;
                    const int64_t vo = (int64_t)(act ? cam : 0) * kVec + row;
                    const double pr = act ? P.p[vo] : 0.0;
                    double bp = 0.0;
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
                        const double pc = __shfl_sync(full, pr, my_sub * 9 + c);
                        if (act) bp += P.Bd[81 * (int64_t)cam + row * 9 + c] * pc;
                    }
                    if (act) {
                        const double qv = bp - (double)ldcg(acc + vo);
                        P.q[vo] = qv;
                        pq += pr * qv;
                        stcg(acc_next + vo, T(0));
                    }
                }
                const double s = block_sum(pq, sb);
                if (threadIdx.x == 0) stcg(part_pq + blockIdx.x, s);
            }
            if (!(ok = barrier())) break;
            const double pq = sum_parts(part_pq, G, sb);
            if (!(pq > 0.0) || !isfinite(pq)) break;
            const double alpha = rho / pq;
            // phase X: x += alpha p; r -= alpha q; z = B~^-1 r
            {
                double rr = 0.0, rz = 0.0;
                for (int w = blockIdx.x * nwarp + wid; w < ncw; w += G * nwarp) {
                    const int cam = w * 3 + my_sub;
                    const bool act = lane < 27 && cam < P.nc;
                    const int64_t vo = (int64_t)(act ? cam : 0) * kVec + row;
                    double rv = 0.0;
                    if (act) {
                        P.x[vo] = fma(alpha, P.p[vo], P.x[vo]);
                        rv = fma(-alpha, P.q[vo], P.r[vo]);
                        P.r[vo] = rv;
                    }
                    double z = 0.0;
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
                        const double rc = __shfl_sync(full, rv, my_sub * 9 + c);
                        if (act) z += P.Binv[81 * (int64_t)cam + row * 9 + c] * rc;
                    }
                    if (act) {
                        P.z[vo] = z;
                        rr += rv * rv;
                        rz += rv * z;
                    }
                }
                const double s_rr = block_sum(rr, sb);
                const double s_rz = block_sum(rz, sb);
                if (threadIdx.x == 0) {
                    stcg(part_rr + blockIdx.x, s_rr);
                    stcg(part_rho + blockIdx.x, s_rz);
                }
            }
            if (!(ok = barrier())) break;
            ++n;
            rho_prev = rho;
            rn = sqrt(sum_parts(part_rr, G, sb));
            if (rn <= tol * r0 || n >= max_iter) break;
        }
    }
    if (!ok) atomicCAS(&st->err, 0, (int)MBA_ERR_TIMEOUT);
    if (ok && blockIdx.x == 0 && threadIdx.x == 0) {
        st->pcg_iters = n;
        st->pcg_rel_res = r0 > 0.0 ? rn / r0 : 0.0;
    }
}

// ---------------------------------------------------------------------------
// back-substitution dp_j = C~_j^-1 (w_j - sum_k Jp~_k^T Jc~_k dc_i(k)) (Eq. 4),
// candidate points, and the model decrease sum_k (-e~_k.d_k - |d_k|^2/2)
// with d_k = Jc~_k dc + Jp~_k dp.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) backsub_kernel(Prob P, double *partial) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sl = reinterpret_cast<T *>(smem_raw);
    __shared__ double sb[kWarps];
    if (P.st->done) return;
    const T *__restrict__ J = (const T *)P.J;
    const T *__restrict__ res = (const T *)P.res;
    const T *__restrict__ Cinv = (const T *)P.Cinv;
    const int cap = P.cap;
    const int64_t npad = P.npad;
    double ldec = 0.0;
    for (int c = blockIdx.x; c < P.n_pchunks; c += gridDim.x) {
        const int j0 = P.pchunk[c], j1 = P.pchunk[c + 1];
        if (j0 == j1) continue;
        const int o0 = P.pt_ptr[j0], m = P.pt_ptr[j1] - o0;
        for (int k = threadIdx.x; k < m; k += kBlock) {
            const int64_t o = (int64_t)o0 + k;
            const int cam = P.pm_cam[o];
            T Jc[18], Jp[6];
            load_jac(J, npad, o, Jc, Jp);
            const double *xc = P.x + (int64_t)cam * kVec;
            T t0 = T(0), t1 = T(0);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const T xa = (T)xc[a];
                t0 += Jc[a] * xa;
                t1 += Jc[9 + a] * xa;
            }
            sl[0 * cap + k] = Jp[0] * t0 + Jp[3] * t1;
            sl[1 * cap + k] = Jp[1] * t0 + Jp[4] * t1;
            sl[2 * cap + k] = Jp[2] * t0 + Jp[5] * t1;
        }
        __syncthreads();
        for (int j = j0 + threadIdx.x; j < j1; j += kBlock) {
            const int b = P.pt_ptr[j] - o0, e = P.pt_ptr[j + 1] - o0;
            T a0 = T(0), a1 = T(0), a2 = T(0);
            for (int s = b; s < e; ++s) {
                a0 += sl[s];
                a1 += sl[cap + s];
                a2 += sl[2 * cap + s];
            }
            const T t0 = (T)P.w[3 * (int64_t)j] - a0, t1 = (T)P.w[3 * (int64_t)j + 1] - a1,
                    t2 = (T)P.w[3 * (int64_t)j + 2] - a2;
            T d[3];
            sym3_apply(Cinv + 6 * (int64_t)j, t0, t1, t2, d);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                P.dp[3 * (int64_t)j + q] = (double)d[q];
                P.pts_new[3 * (int64_t)j + q] = P.pts[3 * (int64_t)j + q] + (double)d[q];
            }
            for (int s = b; s < e; ++s) {
                sl[s] = d[0];
                sl[cap + s] = d[1];
                sl[2 * cap + s] = d[2];
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += kBlock) {
            const int64_t o = (int64_t)o0 + k;
            const int cam = P.pm_cam[o];
            T Jc[18], Jp[6];
            load_jac(J, npad, o, Jc, Jp);
            const double *xc = P.x + (int64_t)cam * kVec;
            T d0 = Jp[0] * sl[k] + Jp[1] * sl[cap + k] + Jp[2] * sl[2 * cap + k];
            T d1 = Jp[3] * sl[k] + Jp[4] * sl[cap + k] + Jp[5] * sl[2 * cap + k];
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const T xa = (T)xc[a];
                d0 += Jc[a] * xa;
                d1 += Jc[9 + a] * xa;
            }
            const double e0 = (double)res[o], e1 = (double)res[npad + o];
            const double dd0 = (double)d0, dd1 = (double)d1;
            ldec += -(e0 * dd0 + e1 * dd1) - 0.5 * (dd0 * dd0 + dd1 * dd1);
        }
        __syncthreads();
    }
    const double s = block_sum(ldec, sb);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
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

bool g_pcg_attr[2] = {false, false};

}  // namespace

cudaError_t launch_damp(const Prob &P, int damping, cudaStream_t s) {
    damp_cameras_kernel<<<(P.nc + 127) / 128, 128, 0, s>>>(P, damping);
    const int64_t nb = (P.np + kBlock - 1) / kBlock;
    const unsigned g = (unsigned)(nb > 152 * 16 ? 152 * 16 : nb);
    if (P.fp32) damp_points_kernel<float><<<g, kBlock, 0, s>>>(P, damping);
    else damp_points_kernel<double><<<g, kBlock, 0, s>>>(P, damping);
    return cudaGetLastError();
}

// Shared-memory plan: the search direction is copied into shared memory once
// per pass when it fits in a third of an SM (so three CTAs stay resident).
void plan_pcg_smem(Prob &P) {
    const int w = P.fp32 ? 4 : 8;
    const int64_t psb = (int64_t)P.nc * 9 * w;
    P.pcg_use_ps = psb <= 72 * 1024 ? 1 : 0;
    P.pcg_smem = P.pcg_use_ps ? (int)psb : 0;
}

int pcg_grid_size(const Prob &P) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)P.pcg_smem;
    int blocks = 0;
    if (P.fp32) {
        cudaFuncSetAttribute(pcg_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, pcg_kernel<float>, kPcgBlock, smem);
    } else {
        cudaFuncSetAttribute(pcg_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, pcg_kernel<double>, kPcgBlock, smem);
    }
    if (blocks < 1) blocks = 1;
    return sms * blocks;
}

cudaError_t launch_pcg(const Prob &P, int mode, int max_iter, double tol, long long spin_limit, int grid,
                       cudaStream_t s) {
    const size_t smem = (size_t)P.pcg_smem;
    // the barrier targets count arrivals from zero in every launch
    cudaError_t e = cudaMemsetAsync(&P.st->barrier, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    Prob Pc = P;
    void *args[] = {(void *)&Pc, (void *)&mode, (void *)&max_iter, (void *)&tol, (void *)&spin_limit};
    if (P.fp32)
        return cudaLaunchCooperativeKernel((const void *)pcg_kernel<float>, dim3(grid), dim3(kPcgBlock), args, smem, s);
    return cudaLaunchCooperativeKernel((const void *)pcg_kernel<double>, dim3(grid), dim3(kPcgBlock), args, smem, s);
}

cudaError_t launch_backsub(const Prob &P, double *partial, int nb, cudaStream_t s) {
    const size_t smem = (P.fp32 ? sizeof(float) : sizeof(double)) * 3 * (size_t)P.cap;
    if (P.fp32) {
        if (!g_pcg_attr[0]) {
            cudaFuncSetAttribute(backsub_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 4 * 2048);
            g_pcg_attr[0] = true;
        }
        backsub_kernel<float><<<nb, kBlock, smem, s>>>(P, partial);
    } else {
        if (!g_pcg_attr[1]) {
            cudaFuncSetAttribute(backsub_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 8 * 2048);
            g_pcg_attr[1] = true;
        }
        backsub_kernel<double><<<nb, kBlock, smem, s>>>(P, partial);
    }
    ldec_final_kernel<<<1, kBlock, 0, s>>>(partial, nb, P.st);
    cams_new_kernel<<<(P.nc * 9 + kBlock - 1) / kBlock, kBlock, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace mba
