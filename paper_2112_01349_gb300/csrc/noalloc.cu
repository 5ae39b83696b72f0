// noalloc.cu -- the bundle-adjustment cost F = 1/2 sum rho(|e_k|^2) for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a framework which
// owns every device allocation through its own pool, real-time loops where an
// allocation (and the implicit synchronisation it can cause) is not allowed,
// and code that must not fail for lack of memory after start-up.  They already
// hold their cameras, points and observations in device memory and only need
// the cost.  mba_problem_create sizes a private pool, so it is not usable
// there; this entry point takes the caller's device arrays and keeps its
// scratch (per-camera rotation tables and per-block partial sums) in a fixed,
// file-scope device array instead.
//
// The scratch array exists once per device that loads the library and stays
// allocated until the process exits.  Every call on a device shares it and
// leaves its contents behind; nothing in it needs to start at zero (each call
// writes the table rows and the partial sums it then reads).  Two calls whose
// work overlaps on the GPU (different streams, no ordering between them) race
// on the scratch and may return wrong costs.
#include <mutex>

#include "mba_internal.cuh"

namespace mba {
namespace {

constexpr int kNaMaxCameras = 8192;  // largest nc this entry point accepts
constexpr int kNaBlocks = 1024;      // cost blocks (one partial sum each)
constexpr size_t kNaTableDoubles = (size_t)kNaMaxCameras * kCamTab;
constexpr size_t kNaScratchDoubles = kNaTableDoubles + kNaBlocks;  // about 1.8 MB

static __device__ __align__(256) double g_na_scratch[kNaScratchDoubles];

// Device address of g_na_scratch per device, found once with that device current.
std::mutex g_na_mu;
double *g_na_addr[256] = {};

__global__ void na_tables_kernel(const double *__restrict__ cams, int32_t nc, double *__restrict__ tab) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        double row[kCamTab];
        camera_table_row(cams + 9 * (int64_t)i, row);
#pragma unroll
        for (int q = 0; q < kCamTab; ++q) tab[(int64_t)i * kCamTab + q] = row[q];
    }
}

// One partial sum of rho(|e_k|^2) per block over the caller's observation order.
// An index out of range makes the block's partial (and so the cost) NaN.
__global__ void __launch_bounds__(kBlock) na_partial_kernel(const double *__restrict__ tab, const double *__restrict__ pts,
                                                            const double *__restrict__ obs,
                                                            const int32_t *__restrict__ ci,
                                                            const int32_t *__restrict__ pi, int32_t nc, int32_t np,
                                                            int64_t n, int loss, double delta,
                                                            double *__restrict__ partial) {
    __shared__ double sred[kWarps];
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int c = ci[k], p = pi[k];
        if (c < 0 || c >= nc || p < 0 || p >= np) {
            acc += __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        double e[2];
        project<double, false>(tab + (int64_t)c * kCamTab, pts[3 * (int64_t)p], pts[3 * (int64_t)p + 1],
                               pts[3 * (int64_t)p + 2], obs[2 * k], obs[2 * k + 1], e, nullptr, nullptr);
        double rho, w;
        loss_weight<double>(loss, delta, e[0] * e[0] + e[1] * e[1], &rho, &w);
        acc += rho;
    }
    const double s = block_sum(acc, sred);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void na_final_kernel(const double *__restrict__ partial, int nb, double *__restrict__ out) {
    __shared__ double sred[kWarps];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    const double s = block_sum(acc, sred);
    if (threadIdx.x == 0) *out = 0.5 * s;
}

}  // namespace
}  // namespace mba

using namespace mba;

extern "C" mba_status mba_cost_noalloc(const double *d_cameras, int32_t nc, const double *d_points, int32_t np,
                                       const double *d_observations, const int32_t *d_cam_idx,
                                       const int32_t *d_pt_idx, int64_t n, int32_t loss, double huber_delta,
                                       double *d_cost, void *cuda_stream) {
    if (!d_cameras || !d_points || !d_observations || !d_cam_idx || !d_pt_idx || !d_cost) return MBA_ERR_INVALID_ARG;
    if (nc < 1 || np < 1 || n < 1) return MBA_ERR_INVALID_ARG;
    if (kUserEdge) return MBA_ERR_INVALID_ARG;  // the BAL camera's cost only
    if (nc > kNaMaxCameras) return MBA_ERR_INVALID_ARG;  // beyond the fixed scratch
    if (loss != MBA_LOSS_NONE && loss != MBA_LOSS_HUBER) return MBA_ERR_INVALID_ARG;
    if (loss == MBA_LOSS_HUBER && !(huber_delta > 0.0)) return MBA_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return MBA_ERR_CUDA;
    double *scratch = nullptr;
    {
        // first call on this device: look up the array's device address (no allocation)
        std::lock_guard<std::mutex> lock(g_na_mu);
        if (!g_na_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return MBA_ERR_CUDA;
            }
            g_na_addr[dev] = (double *)p;
        }
        scratch = g_na_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *tab = scratch, *partial = scratch + kNaTableDoubles;
    int64_t nb = (n + kBlock - 1) / kBlock;
    if (nb > kNaBlocks) nb = kNaBlocks;
    na_tables_kernel<<<(nc + 127) / 128, 128, 0, s>>>(d_cameras, nc, tab);
    na_partial_kernel<<<(unsigned)nb, kBlock, 0, s>>>(tab, d_points, d_observations, d_cam_idx, d_pt_idx, nc, np, n,
                                                     loss, huber_delta, partial);
    na_final_kernel<<<1, kBlock, 0, s>>>(partial, (int)nb, d_cost);
    return cudaGetLastError() == cudaSuccess ? MBA_OK : MBA_ERR_CUDA;
}
