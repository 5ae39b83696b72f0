/* mba_jet.cuh -- forward-mode automatic differentiation for edge functors.
 *
 * The paper's automatic-differentiation path (Sec. 3.2, the JetVector; the
 * "-a" rows of its timing tables) evaluates the edge's residual function on
 * dual numbers, so the Jacobian of a user-defined edge follows from code that
 * computes only the residual.  This header gives the same capability for
 * device (and host) code:
 *
 *   mba::Jet<T, N>   a value with N partial derivatives, held in registers;
 *                    +, -, *, / and ad_sqrt, ad_sin, ad_cos, ad_sincos follow
 *                    the chain rule (the ad_ functions also take plain T).
 *   mba::jet_jacobian<K, CAM, PT>(f, cam, pt, val, Jc, Jp)
 *                    evaluates an edge functor f once per K seeded directions
 *                    and returns its value and the requested Jacobian blocks.
 *
 * An edge functor maps one camera block (kCam parameters) and one point block
 * (kPt parameters) to the predicted measurement (kOut values), templated on the
 * scalar type S so that the same code runs on T and on Jet<T, K>:
 *
 *   struct MyEdge {
 *       static constexpr int kCam = 9, kPt = 3, kOut = 2;
 *       template <class S> MBA_HD void operator()(const S *cam, const S *pt, S *out) const;
 *   };
 *
 * The paper's JetVector stores every jet component as a device-wide vector and
 * runs one kernel per arithmetic operation.  Here one thread evaluates the
 * whole functor on register-resident jets, and the K partials of each pass
 * are the register-pressure knob: K = kCam + kPt is one pass, smaller K trades
 * registers for repeated passes.  The header is plain C++ when compiled
 * without nvcc (host tests).
 */
#pragma once

#ifdef __CUDACC__
#define MBA_HD __host__ __device__ __forceinline__
#else
#define MBA_HD inline
#include <cmath>
#endif

namespace mba {

// Math with one spelling for T and Jet<T, N>, on the device and the host
// (ad_ names, so that they never compete with the C library's overloads).
MBA_HD float ad_sqrt(float x) {
#ifdef __CUDA_ARCH__
    return ::sqrtf(x);
#else
    return std::sqrt(x);
#endif
}
MBA_HD double ad_sqrt(double x) {
#ifdef __CUDA_ARCH__
    return ::sqrt(x);
#else
    return std::sqrt(x);
#endif
}
MBA_HD void ad_sincos(float x, float *s, float *c) {
#ifdef __CUDA_ARCH__
    ::sincosf(x, s, c);
#else
    *s = std::sin(x);
    *c = std::cos(x);
#endif
}
MBA_HD void ad_sincos(double x, double *s, double *c) {
#ifdef __CUDA_ARCH__
    ::sincos(x, s, c);
#else
    *s = std::sin(x);
    *c = std::cos(x);
#endif
}
MBA_HD float ad_sin(float x) {
    float s, c;
    ad_sincos(x, &s, &c);
    return s;
}
MBA_HD double ad_sin(double x) {
    double s, c;
    ad_sincos(x, &s, &c);
    return s;
}
MBA_HD float ad_cos(float x) {
    float s, c;
    ad_sincos(x, &s, &c);
    return c;
}
MBA_HD double ad_cos(double x) {
    double s, c;
    ad_sincos(x, &s, &c);
    return c;
}
template <typename T>
MBA_HD T value_of(T x) {
    return x;
}

// ---------------------------------------------------------------------------
// Dual number: a + sum_i v[i] eps_i with eps_i eps_j = 0.
// ---------------------------------------------------------------------------
template <typename T, int N>
struct Jet {
    T a;
    T v[N];

    MBA_HD Jet() : a(T(0)) {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = T(0);
    }
    MBA_HD Jet(T x) : a(x) {  // a constant
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = T(0);
    }
    MBA_HD Jet(T x, int k) : a(x) {  // the k-th seeded variable (k outside [0, N): a constant)
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = i == k ? T(1) : T(0);
    }
};

template <typename T, int N>
MBA_HD T value_of(const Jet<T, N> &x) {
    return x.a;
}

template <typename T, int N>
MBA_HD Jet<T, N> operator+(const Jet<T, N> &x, const Jet<T, N> &y) {
    Jet<T, N> r;
    r.a = x.a + y.a;
#pragma unroll
    for (int i = 0; i < N; ++i) r.v[i] = x.v[i] + y.v[i];
    return r;
}
template <typename T, int N>
MBA_HD Jet<T, N> operator-(const Jet<T, N> &x, const Jet<T, N> &y) {
    Jet<T, N> r;
    r.a = x.a - y.a;
#pragma unroll
    for (int i = 0; i < N; ++i) r.v[i] = x.v[i] - y.v[i];
    return r;
}
template <typename T, int N>
MBA_HD Jet<T, N> operator-(const Jet<T, N> &x) {
    Jet<T, N> r;
    r.a = -x.a;
#pragma unroll
    for (int i = 0; i < N; ++i) r.v[i] = -x.v[i];
    return r;
}
// product rule: d(xy) = y dx + x dy
template <typename T, int N>
MBA_HD Jet<T, N> operator*(const Jet<T, N> &x, const Jet<T, N> &y) {
    Jet<T, N> r;
    r.a = x.a * y.a;
#pragma unroll
    for (int i = 0; i < N; ++i) r.v[i] = y.a * x.v[i] + x.a * y.v[i];
    return r;
}
// quotient rule: d(x/y) = (dx - (x/y) dy) / y
template <typename T, int N>
MBA_HD Jet<T, N> operator/(const Jet<T, N> &x, const Jet<T, N> &y) {
    Jet<T, N> r;
    const T iy = T(1) / y.a;
    r.a = x.a * iy;
#pragma unroll
    for (int i = 0; i < N; ++i) r.v[i] = (x.v[i] - r.a * y.v[i]) * iy;
    return r;
}
// mixed jet / scalar forms
template <typename T, int N>
MBA_HD Jet<T, N> operator+(const Jet<T, N> &x, T s) {
    Jet<T, N> r = x;
    r.a = x.a + s;
    return r;
}
template <typename T, int N>
MBA_HD Jet<T, N> operator+(T s, const Jet<T, N> &x) {
    return x + s;
}
template <typename T, int N>
MBA_HD Jet<T, N> operator-(const Jet<T, N> &x, T s) {
    Jet<T, N> r = x;
    r.a = x.a - s;
    return r;
}
template <typename T, int N>
MBA_HD Jet<T, N> operator-(T s, const Jet<T, N> &x) {
    Jet<T, N> r;
    r.a = s - x.a;
#pragma unroll
    for (int i = 0; i < N; ++i) r.v[i] = -x.v[i];
    return r;
}
template <typename T, int N>
MBA_HD Jet<T, N> operator*(const Jet<T, N> &x, T s) {
    Jet<T, N> r;
    r.a = x.a * s;
#pragma unroll
    for (int i = 0; i < N; ++i) r.v[i] = x.v[i] * s;
    return r;
}
template <typename T, int N>
MBA_HD Jet<T, N> operator*(T s, const Jet<T, N> &x) {
    return x * s;
}
template <typename T, int N>
MBA_HD Jet<T, N> operator/(const Jet<T, N> &x, T s) {
    return x * (T(1) / s);
}
template <typename T, int N>
MBA_HD Jet<T, N> operator/(T s, const Jet<T, N> &y) {  // d(s/y) = -(s/y) dy / y
    Jet<T, N> r;
    const T iy = T(1) / y.a;
    r.a = s * iy;
#pragma unroll
    for (int i = 0; i < N; ++i) r.v[i] = -r.a * y.v[i] * iy;
    return r;
}
template <typename T, int N>
MBA_HD Jet<T, N> &operator+=(Jet<T, N> &x, const Jet<T, N> &y) {
    x = x + y;
    return x;
}
template <typename T, int N>
MBA_HD Jet<T, N> &operator-=(Jet<T, N> &x, const Jet<T, N> &y) {
    x = x - y;
    return x;
}
template <typename T, int N>
MBA_HD Jet<T, N> &operator*=(Jet<T, N> &x, const Jet<T, N> &y) {
    x = x * y;
    return x;
}
// comparisons look at the value only (branches of the functor)
template <typename T, int N>
MBA_HD bool operator<(const Jet<T, N> &x, T s) {
    return x.a < s;
}
template <typename T, int N>
MBA_HD bool operator>(const Jet<T, N> &x, T s) {
    return x.a > s;
}

// d sqrt(x) = dx / (2 sqrt(x))
template <typename T, int N>
MBA_HD Jet<T, N> ad_sqrt(const Jet<T, N> &x) {
    Jet<T, N> r;
    r.a = ad_sqrt(x.a);
    const T h = T(0.5) / r.a;
#pragma unroll
    for (int i = 0; i < N; ++i) r.v[i] = x.v[i] * h;
    return r;
}
// d sin(x) = cos(x) dx, d cos(x) = -sin(x) dx
template <typename T, int N>
MBA_HD void ad_sincos(const Jet<T, N> &x, Jet<T, N> *s, Jet<T, N> *c) {
    T sa, ca;
    ad_sincos(x.a, &sa, &ca);
    s->a = sa;
    c->a = ca;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        s->v[i] = ca * x.v[i];
        c->v[i] = -sa * x.v[i];
    }
}
template <typename T, int N>
MBA_HD Jet<T, N> ad_sin(const Jet<T, N> &x) {
    Jet<T, N> s, c;
    ad_sincos(x, &s, &c);
    return s;
}
template <typename T, int N>
MBA_HD Jet<T, N> ad_cos(const Jet<T, N> &x) {
    Jet<T, N> s, c;
    ad_sincos(x, &s, &c);
    return c;
}

// ---------------------------------------------------------------------------
// Edge value and Jacobians by forward mode.  The parameter vector is the
// camera block followed by the point block (F::kCam + F::kPt directions);
// each pass seeds K consecutive directions of the requested blocks (CAM, PT)
// and reads K columns of the Jacobian.  Jc is kOut x kCam and Jp is
// kOut x kPt, row major; a block that is not requested is left untouched.
// ---------------------------------------------------------------------------
template <int K, bool CAM, bool PT, class F, typename T>
MBA_HD void jet_jacobian(const F &f, const T *cam, const T *pt, T *val, T *Jc, T *Jp) {
    constexpr int NC = F::kCam, NP = F::kPt, NO = F::kOut;
    constexpr int d0 = CAM ? 0 : NC, d1 = PT ? NC + NP : NC;
    if (d0 >= d1) {
        f(cam, pt, val);
        return;
    }
#pragma unroll
    for (int base = d0; base < d1; base += K) {
        Jet<T, K> jc[NC], jp[NP], out[NO];
#pragma unroll
        for (int i = 0; i < NC; ++i) jc[i] = Jet<T, K>(cam[i], i - base);
#pragma unroll
        for (int i = 0; i < NP; ++i) jp[i] = Jet<T, K>(pt[i], NC + i - base);
        f(jc, jp, out);
#pragma unroll
        for (int r = 0; r < NO; ++r) {
            val[r] = out[r].a;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int d = base + k;
                if (d >= d1) continue;
                if (d < NC) Jc[r * NC + d] = out[r].v[k];
                else Jp[r * NP + (d - NC)] = out[r].v[k];
            }
        }
    }
}

}  // namespace mba
