// api.cu -- host side of the C ABI declared in include/mba.h: problem creation
// (one device pool sized up front), the solve driver that issues the LM
// iterations without host round trips, and the inspection entry points.
#include <cstdio>
#include <cstring>
#include <atomic>
#include <string>
#include <vector>

#include "mba_internal.cuh"


using namespace mba;

namespace {

thread_local std::string g_err;

constexpr int kTraceCap = 4096;
constexpr int64_t kEvalSlice = 1 << 18;
constexpr long long kDefaultSpin = 4000000;

mba_status fail(mba_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(MBA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

size_t al(size_t v) { return (v + 255) & ~size_t(255); }

struct Carve {
    char *base = nullptr;
    size_t off = 0;
    template <typename X>
    X *take(size_t count) {
        X *p = base ? reinterpret_cast<X *>(base + off) : nullptr;
        off += al(sizeof(X) * (count ? count : 1));
        return p;
    }
};

}  // namespace

namespace mba {
// process-wide cap on the device memory one creation may allocate (0 = none)
static std::atomic<unsigned long long> g_mem_limit{0};
bool over_memory_limit(size_t bytes) {
    const unsigned long long l = g_mem_limit.load();
    return l != 0 && (unsigned long long)bytes > l;
}
mba_status api_fail(mba_status st, const char *msg) {
    g_err = msg ? msg : "";
    return st;
}
}  // namespace mba

struct mba_problem {
    Prob P;
    cudaStream_t stream = nullptr;
    void *pool = nullptr;
    size_t pool_bytes = 0;
    int32_t *cfirst = nullptr;      // per camera first chunk (device)
    int32_t *orig_cam = nullptr, *orig_pt = nullptr;
    double2 *orig_uv = nullptr;
    double *eval_stage = nullptr;   // kEvalSlice x 26 doubles
    double *part_a = nullptr, *part_b = nullptr;
    double *scalar = nullptr;       // 8 doubles of scratch results
    int nb_chunk = 0, nb_cost = 0;
    int pcg_grid = 0;
    mba_iteration *trace_dev = nullptr;
    double last_mu = -1.0;  // damping of the last accepted step of the last solve
};

extern "C" {

void mba_problem_options_default(mba_problem_options *o) {
    if (!o) return;
    o->precision = MBA_FP64;
    o->loss = MBA_LOSS_NONE;
    o->huber_delta = 0.0;
    o->cuda_stream = nullptr;
    o->jacobian = MBA_JACOBIAN_ANALYTIC;
    o->pad = 0;
}

void mba_solver_options_default(mba_solver_options *o) {
    if (!o) return;
    o->max_iter = 10;
    o->pcg_max_iter = 100;
    o->pcg_rel_tol = 1e-10;
    o->damping = MBA_DAMP_DIAG;
    o->initial_radius = 1e4;
    o->min_relative_decrease = 1e-3;
    o->function_tol = 0.0;
    o->barrier_spin_limit = 0;
    o->collect_timing = 0;
    o->preconditioner = MBA_PRECOND_BLOCK_JACOBI;
    o->forcing = 0;
    o->cost_arithmetic = MBA_COST_FP64;
    o->pcg_variant = MBA_PCG_STANDARD;
}

const char *mba_edge_name(void) { return kUserEdge ? MBA_STR(MBA_EDGE_TYPE) : "BalEdge"; }

const char *mba_status_string(mba_status s) {
    switch (s) {
        case MBA_OK: return "MBA_OK";
        case MBA_ERR_INVALID_ARG: return "MBA_ERR_INVALID_ARG";
        case MBA_ERR_OOM: return "MBA_ERR_OOM";
        case MBA_ERR_CUDA: return "MBA_ERR_CUDA";
        case MBA_ERR_NONFINITE: return "MBA_ERR_NONFINITE";
        case MBA_ERR_TIMEOUT: return "MBA_ERR_TIMEOUT";
        case MBA_ERR_NOT_CONVERGED: return "MBA_ERR_NOT_CONVERGED";
    }
    return "MBA_ERR_UNKNOWN";
}

const char *mba_last_error(void) { return g_err.c_str(); }

mba_status mba_set_device_memory_limit(size_t bytes) {
    mba::g_mem_limit.store((unsigned long long)bytes);
    return MBA_OK;
}

void mba_problem_destroy(mba_problem *pr) {
    if (!pr) return;
    if (pr->stream) cudaStreamSynchronize(pr->stream);
    if (pr->pool) cudaFree(pr->pool);
    delete pr;
}

mba_status mba_problem_create(const double *cameras, int32_t nc, const double *points, int32_t np,
                              const double *observations, const int32_t *cam_idx, const int32_t *pt_idx, int64_t n,
                              const mba_problem_options *opt, mba_problem **out) {
    g_err.clear();
    if (!out) return fail(MBA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cameras || !points || !observations || !cam_idx || !pt_idx)
        return fail(MBA_ERR_INVALID_ARG, "a required input pointer is NULL");
    if (nc < 1 || np < 1 || n < 1) return fail(MBA_ERR_INVALID_ARG, "nc, np and n must be >= 1");
    if (n >= (int64_t(1) << 31) - 4096) return fail(MBA_ERR_INVALID_ARG, "n must be below 2^31 - 4096");
    mba_problem_options o;
    mba_problem_options_default(&o);
    if (opt) o = *opt;
    if (o.precision != MBA_FP64 && o.precision != MBA_FP32_MIXED) return fail(MBA_ERR_INVALID_ARG, "bad precision");
    if (o.loss != MBA_LOSS_NONE && o.loss != MBA_LOSS_HUBER) return fail(MBA_ERR_INVALID_ARG, "bad loss");
    if (o.loss == MBA_LOSS_HUBER && !(o.huber_delta > 0.0)) return fail(MBA_ERR_INVALID_ARG, "huber_delta must be > 0");
    if (o.jacobian != MBA_JACOBIAN_ANALYTIC && o.jacobian != MBA_JACOBIAN_AUTODIFF)
        return fail(MBA_ERR_INVALID_ARG, "bad jacobian source");
    if (kUserEdge && o.jacobian != MBA_JACOBIAN_AUTODIFF)
        return fail(MBA_ERR_INVALID_ARG, "this library evaluates a user edge type: use MBA_JACOBIAN_AUTODIFF");

    mba_problem *pr = new mba_problem();
    Prob &P = pr->P;
    std::memset(&P, 0, sizeof(P));
    pr->stream = (cudaStream_t)o.cuda_stream;
    cudaStream_t s = pr->stream;
    P.nc = nc;
    P.np = np;
    P.n = n;
    P.npad = ((n + 63) / 64) * 64 + 64;
    P.fp32 = o.precision == MBA_FP32_MIXED;
    P.loss = o.loss;
    P.delta = o.huber_delta;
    P.autodiff = o.jacobian == MBA_JACOBIAN_AUTODIFF;
    P.fact = (P.fp32 && !P.autodiff) ? 1 : 0;  // FP32-mixed analytic: the factored Schur product
    const size_t w = P.fp32 ? 4 : 8;
    const int64_t cbound = n / kCamChunk + (int64_t)nc + 2;     // camera chunks
    pr->pcg_grid = 0;
    int sms = 0;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
        if (sms > 4096) sms = 4096;
        pr->nb_chunk = sms * 4;
    }
    pr->nb_cost = cost_grid(P);
    const int red_len = 3 * 8192;
    const int64_t stage = n < kEvalSlice ? n : kEvalSlice;

    auto layout = [&](Carve &c) {
        P.cams = c.take<double>(9 * (size_t)nc);
        P.cams_new = c.take<double>(9 * (size_t)nc);
        P.cams0 = c.take<double>(9 * (size_t)nc);
        P.pts = c.take<double>(3 * (size_t)np);
        P.pts_new = c.take<double>(3 * (size_t)np);
        P.pts0 = c.take<double>(3 * (size_t)np);
        P.pm_cam = c.take<int32_t>(n + 64);  // slack for 16-byte-rounded bulk copies
        P.pm_pt = c.take<int32_t>(n);
        P.pm_orig = c.take<int32_t>(n);
        P.pm_uv = c.take<double2>(n);
        P.pt_ptr = c.take<int32_t>((size_t)np + 64);  // slack for 16-byte-rounded bulk copies
        P.cm_pt = c.take<int32_t>(n);
        P.cm_orig = c.take<int32_t>(n);
        P.cm_uv = c.take<double2>(n);
        P.cam_ptr = c.take<int32_t>((size_t)nc + 1);
        P.wchunk = c.take<int2>((size_t)np + 64);
        P.tiles = c.take<int2>((size_t)np + 2);
        P.tdesc = c.take<int4>(3 * ((size_t)np + 2));
        P.long_chunks = c.take<int32_t>((size_t)np + 2);
        P.cchunk_cam = c.take<int32_t>(cbound);
        P.cchunk_beg = c.take<int32_t>(cbound + 1);
        pr->cfirst = c.take<int32_t>((size_t)nc + 1);
        pr->orig_cam = c.take<int32_t>(n);
        pr->orig_pt = c.take<int32_t>(n);
        pr->orig_uv = c.take<double2>(n);
        P.J = P.fact ? nullptr : c.take<char>(24 * (size_t)P.npad * w);
        P.res = c.take<char>(2 * (size_t)P.npad * w);
        P.camtab = c.take<char>((size_t)nc * kCamTab * w);
        P.camtab64 = c.take<double>((size_t)nc * kCamTab);
        P.Hpp = c.take<double>(45 * (size_t)nc);
        P.v = c.take<double>(9 * (size_t)nc);
        P.Hll = c.take<double>(6 * (size_t)np);
        P.w = c.take<double>(3 * (size_t)np);
        P.cpart = c.take<double>(54 * (size_t)cbound);
        P.Bd = c.take<double>(81 * (size_t)nc);
        P.Binv = c.take<double>(81 * (size_t)nc);
        P.Cinv = c.take<char>((6 * (size_t)np + 64) * w);
        P.x = c.take<double>((size_t)nc * kVec);
        P.r = c.take<double>((size_t)nc * kVec);
        P.z = c.take<double>((size_t)nc * kVec);
        P.p = c.take<double>((size_t)nc * kVec);
        P.q = c.take<double>((size_t)nc * kVec);
        P.g = c.take<double>((size_t)nc * kVec);
        P.pT = c.take<char>((size_t)nc * ((P.fp32 && !P.autodiff) ? kRow * 4 : kVec * w));
        P.p2 = c.take<double>((size_t)nc * kVec);
        P.sbuf = c.take<char>(2 * (size_t)P.npad * w);
        P.cta_cam = c.take<int32_t>(4096 + 1);
        P.pm2cm = c.take<int32_t>(n + 64);
        P.pm_uv32 = P.fp32 ? c.take<float2>(n) : nullptr;
        P.cm_uv32 = P.fp32 ? c.take<float2>(n) : nullptr;
        P.pts32 = P.fp32 ? c.take<float4>((size_t)np) : nullptr;
        P.cam_fixed = c.take<uint8_t>((size_t)nc);
        P.pt_fixed = c.take<uint8_t>((size_t)np);
        // copies for the PCG: the camera-major stored Jacobian (FP64, or FP32-mixed
        // with dual numbers), else the factored form's per-observation data
        const bool fact = P.fact != 0;
        P.PXpm = fact ? c.take<float>(3 * (size_t)P.npad) : nullptr;
        P.Jph = fact ? c.take<float>(6 * (size_t)P.npad) : nullptr;
        P.RXcm = fact ? c.take<float>(4 * (size_t)P.npad) : nullptr;
        P.swpm = (fact && o.loss != MBA_LOSS_NONE) ? c.take<float>((size_t)P.npad) : nullptr;
        P.camff = fact ? c.take<float2>(16 * (size_t)nc) : nullptr;
        P.uvff = fact ? c.take<float4>((size_t)n) : nullptr;
        P.ptsff = fact ? c.take<float2>(3 * (size_t)np) : nullptr;
        // float copies of z and p (the factored form: their camera rows, kRow floats)
        P.zT = P.fp32 ? c.take<float>((size_t)nc * (fact ? kRow : kVec)) : nullptr;
        P.pT2 = c.take<char>((size_t)nc * (fact ? kRow * 4 : kVec * w));
        P.Jcm = P.fp32 ? nullptr : c.take<double>(18 * (size_t)P.npad);
        P.JcmT = P.fp32 ? (P.autodiff ? (void *)c.take<float>(18 * (size_t)P.npad) : nullptr) : (void *)P.Jcm;
        P.dp = c.take<double>(3 * (size_t)np);
        P.red = c.take<double>(red_len);
        pr->part_a = c.take<double>(8192);
        pr->part_b = c.take<double>(8192);
        pr->scalar = c.take<double>(8);
        P.st = c.take<DevState>(1);
        pr->trace_dev = c.take<mba_iteration>(kTraceCap);
        pr->eval_stage = c.take<double>(26 * (size_t)stage);
    };
    Carve sizing;
    layout(sizing);
    pr->pool_bytes = sizing.off;
    P.red_len = red_len;
    const size_t sort_tmp = stable_sort_tmp_bytes(n, np > nc ? np : nc);
    const size_t setup_bytes = sort_tmp + al(sizeof(double) * 2 * (size_t)n) + 256;
    if (mba::over_memory_limit(pr->pool_bytes + setup_bytes)) {
        const size_t need = pr->pool_bytes + setup_bytes;
        delete pr;
        return fail(MBA_ERR_OOM, "device memory limit: creation needs " + std::to_string(need) + " bytes");
    }
    if (cudaMalloc(&pr->pool, pr->pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete pr;
        return fail(MBA_ERR_OOM, "device pool of " + std::to_string(pr->pool_bytes) + " bytes");
    }
    Carve real;
    real.base = (char *)pr->pool;
    layout(real);
    P.cfirst = pr->cfirst;

    // temporary buffers for the set-up only
    void *tmp = nullptr;
    if (cudaMalloc(&tmp, setup_bytes) != cudaSuccess) {
        cudaGetLastError();
        mba_problem_destroy(pr);
        return fail(MBA_ERR_OOM, "set-up scratch");
    }
    double *obs_d = (double *)((char *)tmp + sort_tmp);
    int32_t *flags = (int32_t *)pr->scalar;  // 4 ints

    auto cleanup_fail = [&](mba_status st, const std::string &m) {
        cudaFree(tmp);
        mba_problem_destroy(pr);
        return fail(st, m);
    };
#define CKC(call)                                                                                     \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return cleanup_fail(MBA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

    CKC(cudaMemcpyAsync(P.cams, cameras, sizeof(double) * 9 * (size_t)nc, cudaMemcpyHostToDevice, s));
    CKC(cudaMemcpyAsync(P.pts, points, sizeof(double) * 3 * (size_t)np, cudaMemcpyHostToDevice, s));
    CKC(cudaMemcpyAsync(obs_d, observations, sizeof(double) * 2 * (size_t)n, cudaMemcpyHostToDevice, s));
    CKC(cudaMemcpyAsync(pr->orig_cam, cam_idx, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    CKC(cudaMemcpyAsync(pr->orig_pt, pt_idx, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    CKC(cudaMemsetAsync(P.cam_fixed, 0, (size_t)nc, s));
    CKC(cudaMemsetAsync(P.pt_fixed, 0, (size_t)np, s));
    CKC(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 4, s));
    CKC(validate_inputs(P.cams, nc, P.pts, np, obs_d, pr->orig_cam, pr->orig_pt, n, flags, s));
    int32_t hflags[4];
    CKC(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    CKC(cudaStreamSynchronize(s));
    if (hflags[0] & 1) return cleanup_fail(MBA_ERR_INVALID_ARG, "camera or point index out of range");
    if (hflags[0] & 2) return cleanup_fail(MBA_ERR_NONFINITE, "non-finite camera, point or observation value");

    CKC(stable_sort_by_key(pr->orig_pt, n, np, P.pm_orig, P.pt_ptr, tmp, sort_tmp, s));
    CKC(stable_sort_by_key(pr->orig_cam, n, nc, P.cm_orig, P.cam_ptr, tmp, sort_tmp, s));
    CKC(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 4, s));
    CKC(gather_layout(P, obs_d, pr->orig_cam, pr->orig_pt, nullptr, flags, s));
    // point-major position -> camera-major position, via the inverse of the
    // camera-major permutation (set-up scratch): the point pass writes s there
    CKC(build_pm2cm(P, (int32_t *)tmp, s));
    CKC(launch_split_observations(P, s));  // float-float pixels for the FP32-mixed solve's cost
    // keep the observations in input order too (for mba_evaluate)
    {
        // interleaved copy obs_d (n x 2) -> orig_uv (double2): same bytes
        CKC(cudaMemcpyAsync(pr->orig_uv, obs_d, sizeof(double) * 2 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    }
    std::vector<int32_t> cam_ptr((size_t)nc + 1);
    CKC(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    CKC(cudaMemcpyAsync(cam_ptr.data(), P.cam_ptr, sizeof(int32_t) * ((size_t)nc + 1), cudaMemcpyDeviceToHost, s));
    CKC(cudaStreamSynchronize(s));
    if ((hflags[0] & 4) || (hflags[2] & 4))
        return cleanup_fail(MBA_ERR_INVALID_ARG, "a camera or point has no observations");
    const int max_track = hflags[1];
    if (max_track > kMaxTrack)
        return cleanup_fail(MBA_ERR_INVALID_ARG,
                            "a point has " + std::to_string(max_track) + " observations; at most 1024 are supported");

    // PCG camera partition: one group of whole cameras per CTA (one CTA per SM),
    // cut at the camera boundaries nearest to equal observation counts; then
    // camera chunks (the smallest power-of-two multiple of kCamChunk for which
    // the busiest CTA's chunk sums fit its shared-memory slots)
    {
        const int G = sms;
        std::vector<int32_t> cta((size_t)G + 1);
        cta[0] = 0;
        cta[G] = nc;
        for (int k = 1; k < G; ++k) {
            const int64_t t = (int64_t)k * n / G;
            int32_t lo = cta[k - 1], hi = nc;  // first camera index i >= lo with cam_ptr[i] >= t
            while (lo < hi) {
                const int32_t mid = lo + (hi - lo) / 2;
                if (cam_ptr[mid] < t) lo = mid + 1;
                else hi = mid;
            }
            int32_t i = lo;
            if (i > cta[k - 1] && i <= nc && t - cam_ptr[i - 1] < (int64_t)cam_ptr[i] - t) --i;
            cta[k] = i < cta[k - 1] ? cta[k - 1] : i;
        }
        int chunk = kCamChunk;
        int max_chunks = 0;
        for (;;) {
            max_chunks = 0;
            for (int k = 0; k < G; ++k) {
                int64_t c = 0;
                for (int32_t i = cta[k]; i < cta[k + 1]; ++i) c += (cam_ptr[i + 1] - cam_ptr[i] + chunk - 1) / chunk;
                if (c > max_chunks) max_chunks = (int)c;
            }
            if ((int64_t)max_chunks * 9 * 8 <= 96 * 1024 || chunk >= (1 << 24)) break;
            chunk *= 2;
        }
        P.pcg_max_cta_chunks = max_chunks;
        std::vector<int32_t> ccam, cbeg, cfirst((size_t)nc + 1);
        for (int32_t i = 0; i < nc; ++i) {
            cfirst[i] = (int32_t)ccam.size();
            for (int32_t b = cam_ptr[i]; b < cam_ptr[i + 1]; b += chunk) {
                ccam.push_back(i);
                cbeg.push_back(b);
            }
        }
        cfirst[nc] = (int32_t)ccam.size();
        cbeg.push_back((int32_t)n);
        P.n_cchunks = (int)ccam.size();
        if (P.n_cchunks > cbound) return cleanup_fail(MBA_ERR_INVALID_ARG, "internal: camera chunk bound");
        // chunks are contiguous in the camera-major order: chunk c is [cbeg[c], cbeg[c+1])
        CKC(cudaMemcpyAsync(P.cchunk_cam, ccam.data(), sizeof(int32_t) * ccam.size(), cudaMemcpyHostToDevice, s));
        CKC(cudaMemcpyAsync(P.cchunk_beg, cbeg.data(), sizeof(int32_t) * cbeg.size(), cudaMemcpyHostToDevice, s));
        CKC(cudaMemcpyAsync(pr->cfirst, cfirst.data(), sizeof(int32_t) * cfirst.size(), cudaMemcpyHostToDevice, s));
        CKC(cudaMemcpyAsync(P.cta_cam, cta.data(), sizeof(int32_t) * cta.size(), cudaMemcpyHostToDevice, s));
        CKC(cudaStreamSynchronize(s));  // host vectors go out of scope
    }
    // warp chunks of the PCG point pass: greedy runs of whole points with at
    // most 32 observations; a point with a longer track forms its own chunk
    {
        std::vector<int32_t> pp((size_t)np + 1);
        CKC(cudaMemcpyAsync(pp.data(), P.pt_ptr, sizeof(int32_t) * pp.size(), cudaMemcpyDeviceToHost, s));
        CKC(cudaStreamSynchronize(s));
        std::vector<int2> wc;
        wc.reserve((size_t)np / 4 + 16);
        int32_t p = 0;
        while (p < np) {
            const int32_t o = pp[p];
            int32_t q = p + 1;
            if (pp[p + 1] - o <= 32)
                while (q < np && pp[q + 1] - o <= 32) ++q;
            wc.push_back(make_int2(p, o));
            p = q;
        }
        wc.push_back(make_int2(np, (int32_t)n));
        P.n_wchunks = (int32_t)wc.size() - 1;
        // tiles of the staged point pass: greedy runs of consecutive chunks with at
        // most 32 observations each, within the stage capacity; a chunk of a longer
        // track ends the run and is listed apart
        std::vector<int2> tiles;
        std::vector<int32_t> longs;
        {
            int32_t tb = -1, tobs = 0, tpts = 0;
            auto close = [&](int32_t end) {
                if (tb >= 0) tiles.push_back(make_int2(tb, end));
                tb = -1;
                tobs = tpts = 0;
            };
            for (int32_t k = 0; k < P.n_wchunks; ++k) {
                const int32_t m = wc[k + 1].y - wc[k].y, npts = wc[k + 1].x - wc[k].x;
                if (m > 32) {
                    close(k);
                    longs.push_back(k);
                    continue;
                }
                if (tb >= 0 && (tobs + m > kTileObs || tpts + npts > kTilePts || k - tb + 1 > kTileChunks)) close(k);
                if (tb < 0) tb = k;
                tobs += m;
                tpts += npts;
            }
            close(P.n_wchunks);
        }
        P.n_tiles = (int32_t)tiles.size();
        P.n_long = (int32_t)longs.size();
        // copy ranges of each tile, rounded to 16 bytes: observations [w0.y, w1.y),
        // C~^-1 floats of points [w0.x, w1.x), CSR offsets pt_ptr[w0.x .. w1.x], chunk
        // entries [cb, ce]
        std::vector<int4> tdesc(3 * tiles.size());
        for (size_t t = 0; t < tiles.size(); ++t) {
            const int2 w0 = wc[tiles[t].x], w1 = wc[tiles[t].y];
            tdesc[3 * t] = make_int4(w0.y & ~3, (w1.y + 3) & ~3, (6 * w0.x) & ~3, (6 * w1.x + 3) & ~3);
            tdesc[3 * t + 1] = make_int4(w0.x & ~3, (w1.x + 4) & ~3, tiles[t].x & ~1, (tiles[t].y + 2) & ~1);
            tdesc[3 * t + 2] = make_int4(tiles[t].x, tiles[t].y, 0, 0);
        }
        if (!tiles.empty()) {
            CKC(cudaMemcpyAsync(P.tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, s));
            CKC(cudaMemcpyAsync(P.tdesc, tdesc.data(), sizeof(int4) * tdesc.size(), cudaMemcpyHostToDevice, s));
        }
        if (!longs.empty())
            CKC(cudaMemcpyAsync(P.long_chunks, longs.data(), sizeof(int32_t) * longs.size(), cudaMemcpyHostToDevice, s));
        CKC(cudaMemcpyAsync(P.wchunk, wc.data(), sizeof(int2) * wc.size(), cudaMemcpyHostToDevice, s));
        CKC(cudaStreamSynchronize(s));
    }
    CKC(cudaMemcpyAsync(P.cams0, P.cams, sizeof(double) * 9 * (size_t)nc, cudaMemcpyDeviceToDevice, s));
    CKC(cudaMemcpyAsync(P.pts0, P.pts, sizeof(double) * 3 * (size_t)np, cudaMemcpyDeviceToDevice, s));
    CKC(cudaMemsetAsync(P.st, 0, sizeof(DevState), s));
    if (P.J) CKC(cudaMemsetAsync(P.J, 0, 24 * (size_t)P.npad * w, s));
    CKC(cudaMemsetAsync(P.res, 0, 2 * (size_t)P.npad * w, s));
    CKC(cudaStreamSynchronize(s));
    cudaFree(tmp);
#undef CKC
    plan_pcg_smem(P);
    pr->pcg_grid = pcg_grid_size(P);
    if (pr->pcg_grid != sms) {
        mba_problem_destroy(pr);
        return fail(MBA_ERR_INVALID_ARG, "the PCG kernel does not fit one CTA per SM for this problem shape");
    }
    if (4 * pr->pcg_grid > red_len) {
        mba_problem_destroy(pr);
        return fail(MBA_ERR_INVALID_ARG, "internal: reduction buffer");
    }
    P.trace = pr->trace_dev;
    P.trace_cap = kTraceCap;
    *out = pr;
    return MBA_OK;
}

mba_status mba_problem_info(const mba_problem *pr, int32_t *nc, int32_t *np, int64_t *n, size_t *bytes) {
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    if (nc) *nc = pr->P.nc;
    if (np) *np = pr->P.np;
    if (n) *n = pr->P.n;
    if (bytes) *bytes = pr->pool_bytes;
    return MBA_OK;
}

}  // extern "C"

namespace {

mba_status check_device_state(mba_problem *pr, DevState *hs) {
    CK(cudaMemcpyAsync(hs, pr->P.st, sizeof(DevState), cudaMemcpyDeviceToHost, pr->stream));
    CK(cudaStreamSynchronize(pr->stream));
    if (hs->err == MBA_ERR_TIMEOUT) return fail(MBA_ERR_TIMEOUT, "a grid barrier of the persistent PCG kernel timed out");
    if (hs->err == MBA_ERR_NONFINITE || hs->blockfail)
        return fail(MBA_ERR_NONFINITE, "a damped block is not positive definite");
    if (hs->err != 0) return fail((mba_status)hs->err, "device error");
    return MBA_OK;
}

// linearise at the current parameters with mu, and form the damped blocks
mba_status prepare_step(mba_problem *pr, double mu, int damping, int precond = MBA_PRECOND_BLOCK_JACOBI) {
    Prob &P = pr->P;
    cudaStream_t s = pr->stream;
    CK(launch_state_init(P, 1.0, mu, 0, s));
    CK(launch_camera_tables_forced(P, P.cams, s));
    CK(launch_linearize_impl(P, pr->cfirst, 1, s));
    CK(launch_damp(P, damping, precond, pr->cfirst, s));
    return MBA_OK;
}

bool valid_solver_opts(const mba_solver_options &o) {
    return o.max_iter >= 0 && o.pcg_max_iter >= 0 && o.pcg_rel_tol >= 0.0 &&
           (o.damping == MBA_DAMP_DIAG || o.damping == MBA_DAMP_IDENTITY) && o.initial_radius > 0.0 &&
           o.function_tol >= 0.0 && o.barrier_spin_limit >= 0 &&
           (o.preconditioner == MBA_PRECOND_BLOCK_JACOBI || o.preconditioner == MBA_PRECOND_SCHUR_JACOBI) &&
           (o.forcing == 0 || o.forcing == 1) &&
           (o.cost_arithmetic == MBA_COST_FP64 || o.cost_arithmetic == MBA_COST_FLOAT_FLOAT) &&
           (o.pcg_variant == MBA_PCG_STANDARD || o.pcg_variant == MBA_PCG_SINGLE_REDUCTION);
}

}  // namespace

extern "C" {

mba_status mba_evaluate(mba_problem *pr, double *cost, double *residuals, double *jac_cam, double *jac_pt) {
    g_err.clear();
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    Prob &P = pr->P;
    cudaStream_t s = pr->stream;
    CK(launch_camera_tables_forced(P, P.cams, s));
    if (cost) {
        CK(launch_cost_impl(P, P.pts, pr->part_b, pr->scalar, nullptr, 0, s));
        CK(cudaMemcpyAsync(cost, pr->scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    if (residuals || jac_cam || jac_pt) {
        const int64_t slice = P.n < kEvalSlice ? P.n : kEvalSlice;
        double *e_d = pr->eval_stage, *jc_d = e_d + 2 * slice, *jp_d = jc_d + 18 * slice;
        for (int64_t k0 = 0; k0 < P.n; k0 += slice) {
            const int64_t m = (P.n - k0) < slice ? (P.n - k0) : slice;
            CK(launch_evaluate_slice(P, pr->orig_cam + k0, pr->orig_pt + k0, pr->orig_uv + k0, m, e_d, jc_d, jp_d, s));
            if (residuals) CK(cudaMemcpyAsync(residuals + 2 * k0, e_d, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, s));
            if (jac_cam) CK(cudaMemcpyAsync(jac_cam + 18 * k0, jc_d, sizeof(double) * 18 * m, cudaMemcpyDeviceToHost, s));
            if (jac_pt) CK(cudaMemcpyAsync(jac_pt + 6 * k0, jp_d, sizeof(double) * 6 * m, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
    }
    CK(cudaStreamSynchronize(s));
    return MBA_OK;
}

mba_status mba_get_parameters(const mba_problem *pr, double *cameras, double *points) {
    g_err.clear();
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    const Prob &P = pr->P;
    if (cameras) CK(cudaMemcpyAsync(cameras, P.cams, sizeof(double) * 9 * (size_t)P.nc, cudaMemcpyDeviceToHost, pr->stream));
    if (points) CK(cudaMemcpyAsync(points, P.pts, sizeof(double) * 3 * (size_t)P.np, cudaMemcpyDeviceToHost, pr->stream));
    CK(cudaStreamSynchronize(pr->stream));
    return MBA_OK;
}

mba_status mba_set_parameters(mba_problem *pr, const double *cameras, const double *points) {
    g_err.clear();
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    const Prob &P = pr->P;
    if (cameras) CK(cudaMemcpyAsync(P.cams, cameras, sizeof(double) * 9 * (size_t)P.nc, cudaMemcpyHostToDevice, pr->stream));
    if (points) CK(cudaMemcpyAsync(P.pts, points, sizeof(double) * 3 * (size_t)P.np, cudaMemcpyHostToDevice, pr->stream));
    CK(cudaStreamSynchronize(pr->stream));
    return MBA_OK;
}

mba_status mba_set_fixed(mba_problem *pr, const uint8_t *cam_fixed, const uint8_t *pt_fixed) {
    g_err.clear();
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    Prob &P = pr->P;
    int any = 0;
    if (cam_fixed)
        for (int32_t i = 0; i < P.nc && !any; ++i) any = cam_fixed[i] != 0;
    if (pt_fixed)
        for (int32_t j = 0; j < P.np && !any; ++j) any = pt_fixed[j] != 0;
    if (cam_fixed) CK(cudaMemcpyAsync(P.cam_fixed, cam_fixed, (size_t)P.nc, cudaMemcpyHostToDevice, pr->stream));
    else CK(cudaMemsetAsync(P.cam_fixed, 0, (size_t)P.nc, pr->stream));
    if (pt_fixed) CK(cudaMemcpyAsync(P.pt_fixed, pt_fixed, (size_t)P.np, cudaMemcpyHostToDevice, pr->stream));
    else CK(cudaMemsetAsync(P.pt_fixed, 0, (size_t)P.np, pr->stream));
    CK(cudaStreamSynchronize(pr->stream));
    P.has_fixed = any;
    return MBA_OK;
}

mba_status mba_reset(mba_problem *pr) {
    g_err.clear();
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    const Prob &P = pr->P;
    CK(cudaMemcpyAsync(P.cams, P.cams0, sizeof(double) * 9 * (size_t)P.nc, cudaMemcpyDeviceToDevice, pr->stream));
    CK(cudaMemcpyAsync(P.pts, P.pts0, sizeof(double) * 3 * (size_t)P.np, cudaMemcpyDeviceToDevice, pr->stream));
    CK(cudaStreamSynchronize(pr->stream));
    return MBA_OK;
}

mba_status mba_get_ordering(const mba_problem *pr, int32_t *pt_perm, int32_t *pt_ptr, int32_t *cam_perm,
                            int32_t *cam_ptr) {
    g_err.clear();
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    const Prob &P = pr->P;
    cudaStream_t s = pr->stream;
    if (pt_perm) CK(cudaMemcpyAsync(pt_perm, P.pm_orig, sizeof(int32_t) * P.n, cudaMemcpyDeviceToHost, s));
    if (pt_ptr) CK(cudaMemcpyAsync(pt_ptr, P.pt_ptr, sizeof(int32_t) * ((size_t)P.np + 1), cudaMemcpyDeviceToHost, s));
    if (cam_perm) CK(cudaMemcpyAsync(cam_perm, P.cm_orig, sizeof(int32_t) * P.n, cudaMemcpyDeviceToHost, s));
    if (cam_ptr) CK(cudaMemcpyAsync(cam_ptr, P.cam_ptr, sizeof(int32_t) * ((size_t)P.nc + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MBA_OK;
}

mba_status mba_linear_system(mba_problem *pr, double mu, int32_t damping, double *Hpp, double *v, double *Hll,
                             double *w, double *rhs) {
    g_err.clear();
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    if (!(mu >= 0.0) || (damping != MBA_DAMP_DIAG && damping != MBA_DAMP_IDENTITY))
        return fail(MBA_ERR_INVALID_ARG, "mu must be >= 0 and damping valid");
    Prob &P = pr->P;
    cudaStream_t s = pr->stream;
    mba_status st = prepare_step(pr, mu, damping);
    if (st) return st;
    if (rhs) CK(launch_pcg(P, PCG_RHS_ONLY, 0, 0.0, kDefaultSpin, pr->pcg_grid, s));
    DevState hs;
    st = check_device_state(pr, &hs);
    if (st) return st;
    if (Hpp) {
        std::vector<double> h(45 * (size_t)P.nc);
        CK(cudaMemcpy(h.data(), P.Hpp, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
        for (int32_t i = 0; i < P.nc; ++i)
            for (int a = 0; a < 9; ++a)
                for (int b = 0; b < 9; ++b) Hpp[81 * (size_t)i + a * 9 + b] = h[45 * (size_t)i + sym9(a, b)];
    }
    if (v) CK(cudaMemcpy(v, P.v, sizeof(double) * 9 * (size_t)P.nc, cudaMemcpyDeviceToHost));
    if (Hll) {
        std::vector<double> h(6 * (size_t)P.np);
        CK(cudaMemcpy(h.data(), P.Hll, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
        for (int32_t j = 0; j < P.np; ++j)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Hll[9 * (size_t)j + a * 3 + b] = h[6 * (size_t)j + sym3(a, b)];
    }
    if (w) CK(cudaMemcpy(w, P.w, sizeof(double) * 3 * (size_t)P.np, cudaMemcpyDeviceToHost));
    if (rhs) {
        std::vector<double> g((size_t)P.nc * kVec);
        CK(cudaMemcpy(g.data(), P.g, sizeof(double) * g.size(), cudaMemcpyDeviceToHost));
        for (int32_t i = 0; i < P.nc; ++i)
            for (int a = 0; a < 9; ++a) rhs[9 * (size_t)i + a] = g[(size_t)i * kVec + a];
    }
    return MBA_OK;
}

mba_status mba_schur_matvec(mba_problem *pr, double mu, int32_t damping, const double *x, double *y) {
    g_err.clear();
    if (!pr || !x || !y) return fail(MBA_ERR_INVALID_ARG, "NULL argument");
    if (!(mu >= 0.0) || (damping != MBA_DAMP_DIAG && damping != MBA_DAMP_IDENTITY))
        return fail(MBA_ERR_INVALID_ARG, "mu must be >= 0 and damping valid");
    Prob &P = pr->P;
    cudaStream_t s = pr->stream;
    mba_status st = prepare_step(pr, mu, damping);
    if (st) return st;
    std::vector<double> buf((size_t)P.nc * kVec, 0.0);
    for (int32_t i = 0; i < P.nc; ++i)
        for (int a = 0; a < 9; ++a) buf[(size_t)i * kVec + a] = x[9 * (size_t)i + a];
    CK(cudaMemcpyAsync(P.p, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, s));
    CK(launch_pcg(P, PCG_MATVEC, 0, 0.0, kDefaultSpin, pr->pcg_grid, s));
    DevState hs;
    st = check_device_state(pr, &hs);
    if (st) return st;
    CK(cudaMemcpy(buf.data(), P.q, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost));
    for (int32_t i = 0; i < P.nc; ++i)
        for (int a = 0; a < 9; ++a) y[9 * (size_t)i + a] = buf[(size_t)i * kVec + a];
    return MBA_OK;
}

mba_status mba_step(mba_problem *pr, double mu, const mba_solver_options *opt, double *dc, double *dp,
                    int32_t *pcg_iters, double *model_decrease) {
    g_err.clear();
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    mba_solver_options o;
    mba_solver_options_default(&o);
    if (opt) o = *opt;
    if (!valid_solver_opts(o) || !(mu >= 0.0)) return fail(MBA_ERR_INVALID_ARG, "bad solver options or mu");
    Prob &P = pr->P;
    cudaStream_t s = pr->stream;
    mba_status st = prepare_step(pr, mu, o.damping, o.preconditioner);
    if (st) return st;
    const long long spin = o.barrier_spin_limit > 0 ? o.barrier_spin_limit : kDefaultSpin;
    CK(launch_pcg(P, PCG_SOLVE, o.pcg_max_iter, o.pcg_rel_tol, spin, pr->pcg_grid, s, 0, o.pcg_variant));
    CK(launch_backsub(P, pr->part_a, pr->nb_chunk, s));
    DevState hs;
    st = check_device_state(pr, &hs);
    if (st) return st;
    if (dc) {
        std::vector<double> buf((size_t)P.nc * kVec);
        CK(cudaMemcpy(buf.data(), P.x, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost));
        for (int32_t i = 0; i < P.nc; ++i)
            for (int a = 0; a < 9; ++a) dc[9 * (size_t)i + a] = buf[(size_t)i * kVec + a];
    }
    if (dp) CK(cudaMemcpy(dp, P.dp, sizeof(double) * 3 * (size_t)P.np, cudaMemcpyDeviceToHost));
    if (pcg_iters) *pcg_iters = hs.pcg_iters;
    if (model_decrease) *model_decrease = hs.model_dec;
    return MBA_OK;
}

mba_status mba_solve(mba_problem *pr, const mba_solver_options *opt, mba_summary *summary) {
    g_err.clear();
    if (!pr) return fail(MBA_ERR_INVALID_ARG, "problem is NULL");
    mba_solver_options o;
    mba_solver_options_default(&o);
    if (opt) o = *opt;
    if (!valid_solver_opts(o)) return fail(MBA_ERR_INVALID_ARG, "bad solver options");
    Prob &P = pr->P;
    cudaStream_t s = pr->stream;
    const long long spin = o.barrier_spin_limit > 0 ? o.barrier_spin_limit : kDefaultSpin;
    const bool timing = o.collect_timing != 0;
    const int ne = timing ? 4 * o.max_iter + 2 : 0;
    std::vector<cudaEvent_t> ev(ne);
    for (int i = 0; i < ne; ++i) CK(cudaEventCreate(&ev[i]));
    auto rec = [&](int i) -> cudaError_t { return timing ? cudaEventRecord(ev[i], s) : cudaSuccess; };

    // accept/reject cost: FP64, or float-float on the FP32 pipe when asked for
    // (FP32-mixed analytic problems only: the float-float pixels exist there)
    const bool ff = P.fact != 0 && o.cost_arithmetic == MBA_COST_FLOAT_FLOAT;
    CK(rec(0));
    CK(launch_state_init(P, o.initial_radius, -1.0, 0, s));
    CK(launch_camera_tables(P, P.cams, false, s));
    CK(launch_cost_impl(P, P.pts, pr->part_b, &P.st->cost, &P.st->initial_cost, 1, s, ff));
    for (int it = 0; it < o.max_iter; ++it) {
        CK(rec(1 + 4 * it));
        CK(launch_camera_tables(P, P.cams, true, s));
        CK(launch_linearize_impl(P, pr->cfirst, 0, s));
        CK(rec(2 + 4 * it));
        CK(launch_damp(P, o.damping, o.preconditioner, pr->cfirst, s));
        CK(rec(3 + 4 * it));
        CK(launch_pcg(P, PCG_SOLVE, o.pcg_max_iter, o.pcg_rel_tol, spin, pr->pcg_grid, s, o.forcing, o.pcg_variant));
        CK(rec(4 + 4 * it));
        CK(launch_backsub(P, pr->part_a, pr->nb_chunk, s));
        CK(launch_camera_tables(P, P.cams_new, false, s));
        CK(launch_cost_impl(P, P.pts_new, pr->part_b, &P.st->cost_new, nullptr, 1, s, ff));
        CK(launch_lm_update(P, o, s));
        CK(launch_accept(P, s));
    }
    CK(rec(ne > 0 ? ne - 1 : 0));
    // state_init, camera table, 2 cost kernels; per iteration: camera table, 3
    // linearisation, 2 damping, PCG, 3 back-substitution, camera table, 2 cost,
    // LM update, accept; the factored form adds the camera rows of dc, the
    // float-float cost its point copy before each cost, the Schur-Jacobi
    // preconditioner two damping kernels
    const int fact = P.fact ? 1 : 0, ffc = ff ? 1 : 0;
    const int launches =
        4 + ffc + (15 + fact + ffc + (o.preconditioner == MBA_PRECOND_SCHUR_JACOBI ? 2 : 0)) * o.max_iter;
    DevState hs;
    mba_status st = check_device_state(pr, &hs);
    if (summary) {
        summary->iterations = hs.iter;
        summary->accepted = hs.accepted_total;
        summary->pcg_iters_total = hs.pcg_total;
        summary->status = st;
        summary->initial_cost = hs.initial_cost;
        summary->final_cost = hs.cost;
        summary->final_radius = hs.radius;
        summary->final_mu = 1.0 / hs.radius;
        summary->ms_total = summary->ms_linearize = summary->ms_pcg = summary->ms_other = 0.0;
        summary->kernel_launches = launches;
        if (timing) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[0], ev[ne - 1]);
            summary->ms_total = t;
            double lin = 0, pcg = 0;
            for (int it = 0; it < o.max_iter; ++it) {
                cudaEventElapsedTime(&t, ev[1 + 4 * it], ev[2 + 4 * it]);
                lin += t;
                cudaEventElapsedTime(&t, ev[3 + 4 * it], ev[4 + 4 * it]);
                pcg += t;
            }
            summary->ms_linearize = lin;
            summary->ms_pcg = pcg;
            summary->ms_other = summary->ms_total - lin - pcg;
        }
        if (summary->trace && summary->trace_capacity > 0) {
            int cnt = hs.iter < summary->trace_capacity ? hs.iter : summary->trace_capacity;
            if (cnt > kTraceCap) cnt = kTraceCap;
            if (cnt > 0)
                CK(cudaMemcpy(summary->trace, pr->trace_dev, sizeof(mba_iteration) * cnt, cudaMemcpyDeviceToHost));
        }
    }
    for (int i = 0; i < ne; ++i) cudaEventDestroy(ev[i]);
    if (hs.accepted_total > 0) pr->last_mu = hs.mu_accepted;
    return st;
}

mba_status mba_adjoint(mba_problem *pr, const mba_solver_options *opt, double mu, const double *grad_cameras,
                       const double *grad_points, double *grad_obs, double *grad_init_cam, double *grad_init_pt,
                       int32_t *pcg_iters) {
    g_err.clear();
    if (!pr || !grad_cameras || !grad_points) return fail(MBA_ERR_INVALID_ARG, "NULL argument");
    mba_solver_options o;
    mba_solver_options_default(&o);
    if (opt) o = *opt;
    if (!valid_solver_opts(o)) return fail(MBA_ERR_INVALID_ARG, "bad solver options");
    if (mu < 0.0) mu = pr->last_mu;
    if (!(mu >= 0.0)) return fail(MBA_ERR_INVALID_ARG, "mu < 0 and no accepted step of a previous solve");
    Prob &P = pr->P;
    cudaStream_t s = pr->stream;
    mba_status st = prepare_step(pr, mu, o.damping, o.preconditioner);
    if (st) return st;
    // right-hand side gbar in place of the gradient (v for cameras, w for points)
    CK(cudaMemcpyAsync(P.v, grad_cameras, sizeof(double) * 9 * (size_t)P.nc, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.w, grad_points, sizeof(double) * 3 * (size_t)P.np, cudaMemcpyHostToDevice, s));
    const long long spin = o.barrier_spin_limit > 0 ? o.barrier_spin_limit : kDefaultSpin;
    CK(launch_pcg(P, PCG_SOLVE, o.pcg_max_iter, o.pcg_rel_tol, spin, pr->pcg_grid, s, 0, o.pcg_variant));
    CK(launch_backsub(P, pr->part_a, pr->nb_chunk, s));  // dp = v_p
    DevState hs;
    st = check_device_state(pr, &hs);
    if (st) return st;
    if (grad_obs) {
        const int64_t slice = P.n < kEvalSlice ? P.n : kEvalSlice;
        for (int64_t k0 = 0; k0 < P.n; k0 += slice) {
            const int64_t m = (P.n - k0) < slice ? (P.n - k0) : slice;
            CK(launch_adjoint_obs(P, pr->orig_cam + k0, pr->orig_pt + k0, pr->orig_uv + k0, m, pr->eval_stage, s));
            CK(cudaMemcpyAsync(grad_obs + 2 * k0, pr->eval_stage, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
    }
    if (grad_init_cam || grad_init_pt) {
        CK(launch_adjoint_init(P, o.damping, mu, s));
        if (grad_init_cam)
            CK(cudaMemcpyAsync(grad_init_cam, P.cams_new, sizeof(double) * 9 * (size_t)P.nc, cudaMemcpyDeviceToHost, s));
        if (grad_init_pt)
            CK(cudaMemcpyAsync(grad_init_pt, P.pts_new, sizeof(double) * 3 * (size_t)P.np, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (pcg_iters) *pcg_iters = hs.pcg_iters;
    return MBA_OK;
}

}  // extern "C"
