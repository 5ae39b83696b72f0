// bal_io.cu -- host-side reader and writer of Bundle-Adjustment-in-the-Large
// text files, the problem format of the paper's BAL experiments (Sec. 6).
//
// Layout (whitespace separated):
//   <num_cameras> <num_points> <num_observations>
//   num_observations lines: <camera index> <point index> <x> <y>
//   num_cameras x 9 values: angle-axis w (3), t (3), f, k1, k2
//   num_points x 3 values:  X, Y, Z
// which is exactly the camera model and residual convention of this library.
// No GPU is involved.
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "mba_internal.cuh"

namespace {

using mba::api_fail;

struct Reader {
    std::vector<char> buf;
    const char *p = nullptr;
    const char *end = nullptr;
    int64_t values = 0;  // tokens consumed (for error messages)

    bool load(const char *path) {
        FILE *f = std::fopen(path, "rb");
        if (!f) return false;
        std::fseek(f, 0, SEEK_END);
        const long sz = std::ftell(f);
        std::fseek(f, 0, SEEK_SET);
        if (sz < 0) {
            std::fclose(f);
            return false;
        }
        buf.resize((size_t)sz + 1);
        const size_t got = std::fread(buf.data(), 1, (size_t)sz, f);
        std::fclose(f);
        buf[got] = '\0';
        p = buf.data();
        end = buf.data() + got;
        return true;
    }
    void skip() {
        while (p < end && (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')) ++p;
    }
    bool integer(long long *v) {
        skip();
        if (p >= end) return false;
        char *q = nullptr;
        errno = 0;
        const long long x = std::strtoll(p, &q, 10);
        if (q == p || errno != 0) return false;
        p = q;
        ++values;
        *v = x;
        return true;
    }
    bool real(double *v) {
        skip();
        if (p >= end) return false;
        char *q = nullptr;
        const double x = std::strtod(p, &q);
        if (q == p) return false;
        p = q;
        ++values;
        *v = x;
        return true;
    }
};

mba_status fail(mba_status st, const std::string &msg) { return api_fail(st, msg.c_str()); }

mba_status bad(const Reader &r, const std::string &what) {
    return fail(MBA_ERR_INVALID_ARG, "BAL file: " + what + " (after " + std::to_string(r.values) + " values)");
}

}  // namespace

extern "C" {

mba_status mba_bal_read(const char *path, int32_t *nc, int32_t *np, int64_t *n, double *cameras, double *points,
                        double *observations, int32_t *cam_idx, int32_t *pt_idx) {
    if (!path || !nc || !np || !n) return api_fail(MBA_ERR_INVALID_ARG, "path and size outputs must not be NULL");
    Reader r;
    if (!r.load(path)) return fail(MBA_ERR_INVALID_ARG, std::string("cannot read ") + path);
    long long c = 0, q = 0, m = 0;
    if (!r.integer(&c) || !r.integer(&q) || !r.integer(&m)) return bad(r, "missing header");
    if (c < 1 || q < 1 || m < 1 || c > INT32_MAX || q > INT32_MAX || m >= (int64_t(1) << 31) - 4096)
        return bad(r, "header sizes out of range");
    *nc = (int32_t)c;
    *np = (int32_t)q;
    *n = (int64_t)m;
    if (!cameras || !points || !observations || !cam_idx || !pt_idx) return MBA_OK;  // size query
    bool finite = true;
    for (long long k = 0; k < m; ++k) {
        long long ci = 0, pi = 0;
        double x = 0.0, y = 0.0;
        if (!r.integer(&ci) || !r.integer(&pi) || !r.real(&x) || !r.real(&y))
            return bad(r, "observation " + std::to_string(k) + " is incomplete");
        if (ci < 0 || ci >= c || pi < 0 || pi >= q)
            return bad(r, "observation " + std::to_string(k) + " has an index out of range");
        cam_idx[k] = (int32_t)ci;
        pt_idx[k] = (int32_t)pi;
        observations[2 * k] = x;
        observations[2 * k + 1] = y;
        finite = finite && std::isfinite(x) && std::isfinite(y);
    }
    for (long long k = 0; k < 9 * c; ++k) {
        if (!r.real(&cameras[k])) return bad(r, "camera block " + std::to_string(k / 9) + " is incomplete");
        finite = finite && std::isfinite(cameras[k]);
    }
    for (long long k = 0; k < 3 * q; ++k) {
        if (!r.real(&points[k])) return bad(r, "point " + std::to_string(k / 3) + " is incomplete");
        finite = finite && std::isfinite(points[k]);
    }
    if (!finite) return api_fail(MBA_ERR_NONFINITE, "BAL file: non-finite value");
    return MBA_OK;
}

mba_status mba_bal_write(const char *path, int32_t nc, int32_t np, int64_t n, const double *cameras,
                         const double *points, const double *observations, const int32_t *cam_idx,
                         const int32_t *pt_idx) {
    if (!path || !cameras || !points || !observations || !cam_idx || !pt_idx)
        return api_fail(MBA_ERR_INVALID_ARG, "a required pointer is NULL");
    if (nc < 1 || np < 1 || n < 1) return api_fail(MBA_ERR_INVALID_ARG, "nc, np and n must be >= 1");
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(MBA_ERR_INVALID_ARG, std::string("cannot write ") + path);
    bool ok = std::fprintf(f, "%d %d %lld\n", nc, np, (long long)n) > 0;
    // %.17g: every double is written so that reading it back gives the same bits
    for (int64_t k = 0; k < n && ok; ++k)
        ok = std::fprintf(f, "%d %d %.17g %.17g\n", cam_idx[k], pt_idx[k], observations[2 * k],
                          observations[2 * k + 1]) > 0;
    for (int64_t k = 0; k < 9 * (int64_t)nc && ok; ++k) ok = std::fprintf(f, "%.17g\n", cameras[k]) > 0;
    for (int64_t k = 0; k < 3 * (int64_t)np && ok; ++k) ok = std::fprintf(f, "%.17g\n", points[k]) > 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(MBA_ERR_INVALID_ARG, std::string("write to ") + path + " failed");
    return MBA_OK;
}

}  // extern "C"
