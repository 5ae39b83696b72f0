// sort.cu -- problem set-up on the device: input validation, the stable
// orderings of the observations by point and by camera (the CSR layout of E
// and E^T, Sec. 4.1), the permuted structure-of-arrays copies and the map from
// point-major to camera-major positions.
#include "mba_internal.cuh"

namespace mba {

namespace {

constexpr int kItems = 8;
constexpr int kTile = kBlock * kItems;  // 2048 elements per tile

// ---------------------------------------------------------------------------
// exclusive scan of int32 (sums must stay below 2^31)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_exclusive_scan(int v, int *total, int *swarp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) swarp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int s = lane < kWarps ? swarp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < kWarps) swarp[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const int warp_off = wid > 0 ? swarp[wid - 1] : 0;
    *total = swarp[kWarps - 1];
    __syncthreads();
    return warp_off + inc - v;
}

__global__ void scan_reduce_kernel(const int32_t *in, int64_t n, int32_t *bsum) {
    __shared__ int sw[kWarps];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (base + i < n) s += in[base + i];
    int tot;
    block_exclusive_scan(s, &tot, sw);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void scan_single_kernel(int32_t *a, int64_t n) {
    __shared__ int sw[kWarps];
    int carry = 0;
    for (int64_t t0 = 0; t0 < n; t0 += kTile) {
        const int64_t base = t0 + (int64_t)threadIdx.x * kItems;
        int v[kItems];
        int s = 0;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            v[i] = base + i < n ? a[base + i] : 0;
            s += v[i];
        }
        int tot;
        int off = block_exclusive_scan(s, &tot, sw) + carry;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (base + i < n) a[base + i] = off;
            off += v[i];
        }
        carry += tot;
    }
}

__global__ void scan_apply_kernel(const int32_t *in, int64_t n, const int32_t *bsum, int32_t *out) {
    __shared__ int sw[kWarps];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int v[kItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int tot;
    int off = block_exclusive_scan(s, &tot, sw) + bsum[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (base + i < n) out[base + i] = off;
        off += v[i];
    }
}

// in-place capable exclusive scan; tmp needs ceil(n / kTile) ints
cudaError_t exclusive_scan(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + kTile - 1) / kTile;
    scan_reduce_kernel<<<(unsigned)nb, kBlock, 0, s>>>(in, n, tmp);
    scan_single_kernel<<<1, kBlock, 0, s>>>(tmp, nb);
    scan_apply_kernel<<<(unsigned)nb, kBlock, 0, s>>>(in, n, tmp, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits.  Each pass is stable: inside a tile, warp w
// owns a contiguous run of 256 elements handled in 8 rounds of 32 lanes; the
// rank among equal digits comes from __match_any_sync, earlier rounds and
// lower lanes first, so equal keys keep their input order.
// ---------------------------------------------------------------------------
__global__ void radix_hist_kernel(const int32_t *keys, int64_t n, int shift, int32_t *hist, int ntiles) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kBlock) {
        const int64_t k = base + i;
        if (k < n) atomicAdd(&h[(keys[k] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void radix_scatter_kernel(const int32_t *kin, const int32_t *vin, int64_t n, int shift,
                                     const int32_t *offs, int ntiles, int32_t *kout, int32_t *vout) {
    __shared__ int wc[kWarps * 256];
    for (int i = threadIdx.x; i < kWarps * 256; i += kBlock) wc[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)blockIdx.x * kTile + (int64_t)wid * (32 * kItems);
    const unsigned lt = (1u << lane) - 1u;
    int dig[kItems], pos[kItems], key[kItems], val[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t k = wbase + r * 32 + lane;
        const bool act = k < n;
        int d = 256 + lane;  // unique, never matches a real digit
        key[r] = 0;
        val[r] = 0;
        if (act) {
            key[r] = kin[k];
            val[r] = vin[k];
            d = (key[r] >> shift) & 255;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        const int leader = __ffs(peers) - 1;
        const int basec = act ? wc[wid * 256 + d] : 0;
        __syncwarp();
        if (act && lane == leader) wc[wid * 256 + d] = basec + __popc(peers);
        __syncwarp();
        dig[r] = act ? d : -1;
        pos[r] = basec + rank;
    }
    __syncthreads();
    {
        const int d = threadIdx.x;
        int run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const int c = wc[w * 256 + d];
            wc[w * 256 + d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        if (dig[r] >= 0) {
            const int d = dig[r];
            const int64_t dst = (int64_t)offs[(int64_t)d * ntiles + blockIdx.x] + wc[wid * 256 + d] + pos[r];
            kout[dst] = key[r];
            vout[dst] = val[r];
        }
    }
}

__global__ void iota_copy_kernel(const int32_t *kin, int64_t n, int32_t *kout, int32_t *vout) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        kout[k] = kin[k];
        vout[k] = (int32_t)k;
    }
}

__global__ void count_keys_kernel(const int32_t *keys, int64_t n, int32_t *cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[keys[k]], 1);
}

inline unsigned grid_for(int64_t n) {
    int64_t g = (n + kBlock - 1) / kBlock;
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned)(g < 1 ? 1 : g);
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

// exclusive scan of n int32 for other files (in place allowed); tmp holds
// exclusive_scan_tmp_ints(n) ints
int64_t exclusive_scan_tmp_ints(int64_t n) { return (n + kTile - 1) / kTile + 1; }
cudaError_t exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp, cudaStream_t s) {
    return exclusive_scan(in, out, n, tmp, s);
}

// ints of scan scratch for the larger of the two scans a sort performs
int64_t scan_tmp_count(int64_t n, int32_t nkeys) {
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int64_t scan_n = 256 * ntiles > (int64_t)nkeys + 1 ? 256 * ntiles : (int64_t)nkeys + 1;
    return (scan_n + kTile - 1) / kTile + 1;
}

size_t stable_sort_tmp_bytes(int64_t n, int32_t nkeys) {
    const int64_t ntiles = (n + kTile - 1) / kTile;
    return align_up(sizeof(int32_t) * n) * 3 + align_up(sizeof(int32_t) * 256 * ntiles) +
           align_up(sizeof(int32_t) * scan_tmp_count(n, nkeys)) + align_up(sizeof(int32_t) * (nkeys + 1));
}

cudaError_t stable_sort_by_key(const int32_t *keys_in, int64_t n, int32_t nkeys, int32_t *perm_out,
                               int32_t *ptr_out, void *tmp, size_t tmp_bytes, cudaStream_t s) {
    if (tmp_bytes < stable_sort_tmp_bytes(n, nkeys)) return cudaErrorInvalidValue;
    const int ntiles = (int)((n + kTile - 1) / kTile);
    char *t = (char *)tmp;
    int32_t *ka = (int32_t *)t; t += align_up(sizeof(int32_t) * n);
    int32_t *kb = (int32_t *)t; t += align_up(sizeof(int32_t) * n);
    int32_t *vb = (int32_t *)t; t += align_up(sizeof(int32_t) * n);
    int32_t *hist = (int32_t *)t; t += align_up(sizeof(int32_t) * 256 * (size_t)ntiles);
    int32_t *stmp = (int32_t *)t; t += align_up(sizeof(int32_t) * scan_tmp_count(n, nkeys));
    int32_t *cnt = (int32_t *)t;

    int bits = 0;
    while (bits < 31 && (1ll << bits) < (long long)nkeys) ++bits;
    int32_t *kcur = ka, *vcur = perm_out, *knext = kb, *vnext = vb;
    iota_copy_kernel<<<grid_for(n), kBlock, 0, s>>>(keys_in, n, kcur, vcur);
    for (int shift = 0; shift < bits; shift += 8) {
        radix_hist_kernel<<<ntiles, kBlock, 0, s>>>(kcur, n, shift, hist, ntiles);
        cudaError_t e = exclusive_scan(hist, hist, (int64_t)256 * ntiles, stmp, s);
        if (e != cudaSuccess) return e;
        radix_scatter_kernel<<<ntiles, kBlock, 0, s>>>(kcur, vcur, n, shift, hist, ntiles, knext, vnext);
        int32_t *tk = kcur; kcur = knext; knext = tk;
        int32_t *tv = vcur; vcur = vnext; vnext = tv;
    }
    if (vcur != perm_out) {
        cudaError_t e = cudaMemcpyAsync(perm_out, vcur, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nkeys + 1), s);
    if (e != cudaSuccess) return e;
    count_keys_kernel<<<grid_for(n), kBlock, 0, s>>>(keys_in, n, cnt);
    return exclusive_scan(cnt, ptr_out, (int64_t)nkeys + 1, stmp, s);
}

// ---------------------------------------------------------------------------
// validation: flags[0] |= 1 bad index, 2 non-finite; flags[1..] unused
// ---------------------------------------------------------------------------
namespace {
__global__ void validate_obs_kernel(const double *obs, const int32_t *ci, const int32_t *pi, int64_t n, int32_t nc,
                                    int32_t np, int32_t *flags) {
    int f = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = ci[k], p = pi[k];
        if (c < 0 || c >= nc || p < 0 || p >= np) f |= 1;
        if (!isfinite(obs[2 * k]) || !isfinite(obs[2 * k + 1])) f |= 2;
    }
    if (f) atomicOr(flags, f);
}

__global__ void validate_params_kernel(const double *a, int64_t m, int32_t *flags) {
    int f = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[k])) f |= 2;
    if (f) atomicOr(flags, f);
}
}  // namespace

cudaError_t validate_inputs(const double *cams, int32_t nc, const double *pts, int32_t np, const double *obs,
                            const int32_t *ci, const int32_t *pi, int64_t n, int32_t *flags, cudaStream_t s) {
    validate_obs_kernel<<<grid_for(n), kBlock, 0, s>>>(obs, ci, pi, n, nc, np, flags);
    validate_params_kernel<<<grid_for(9 * (int64_t)nc), kBlock, 0, s>>>(cams, 9 * (int64_t)nc, flags);
    validate_params_kernel<<<grid_for(3 * (int64_t)np), kBlock, 0, s>>>(pts, 3 * (int64_t)np, flags);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// permuted copies and segment statistics
// ---------------------------------------------------------------------------
namespace {
__global__ void gather_kernel(const int32_t *perm, int64_t n, const double *obs, const int32_t *ci,
                              const int32_t *pi, int32_t *o_cam, int32_t *o_pt, double2 *o_uv) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = perm[s];
        if (o_cam) o_cam[s] = ci[k];
        if (o_pt) o_pt[s] = pi[k];
        o_uv[s] = make_double2(obs[2 * (int64_t)k], obs[2 * (int64_t)k + 1]);
    }
}

// flags[0] |= 4 if a segment is empty; flags[1] = max segment length
__global__ void segment_stats_kernel(const int32_t *ptr, int32_t nseg, int32_t *flags) {
    int f = 0, mx = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nseg; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t len = ptr[j + 1] - ptr[j];
        if (len <= 0) f |= 4;
        if (len > mx) mx = len;
    }
    if (f) atomicOr(flags, f);
    atomicMax(flags + 1, mx);
}

}  // namespace

cudaError_t gather_layout(Prob &P, const double *obs_in, const int32_t *ci, const int32_t *pi, int32_t *max_track,
                          int32_t *flags, cudaStream_t s) {
    gather_kernel<<<grid_for(P.n), kBlock, 0, s>>>(P.pm_orig, P.n, obs_in, ci, pi, P.pm_cam, P.pm_pt, P.pm_uv);
    gather_kernel<<<grid_for(P.n), kBlock, 0, s>>>(P.cm_orig, P.n, obs_in, ci, pi, nullptr, P.cm_pt, P.cm_uv);
    segment_stats_kernel<<<grid_for(P.np), kBlock, 0, s>>>(P.pt_ptr, P.np, flags);
    segment_stats_kernel<<<grid_for(P.nc), kBlock, 0, s>>>(P.cam_ptr, P.nc, flags + 2);
    (void)max_track;
    return cudaGetLastError();
}

namespace {
__global__ void invert_perm_kernel(const int32_t *perm, int64_t n, int32_t *inv) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x)
        inv[perm[o]] = (int32_t)o;
}
__global__ void pm2cm_kernel(const int32_t *pm_orig, const int32_t *inv, int64_t n, int32_t *pm2cm) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x)
        pm2cm[o] = inv[pm_orig[o]];
}
}  // namespace

// pm2cm[o] = camera-major position of the observation at point-major position o
cudaError_t build_pm2cm(Prob &P, int32_t *tmp_n, cudaStream_t s) {
    invert_perm_kernel<<<grid_for(P.n), kBlock, 0, s>>>(P.cm_orig, P.n, tmp_n);
    pm2cm_kernel<<<grid_for(P.n), kBlock, 0, s>>>(P.pm_orig, tmp_n, P.n, P.pm2cm);
    return cudaGetLastError();
}


}  // namespace mba
