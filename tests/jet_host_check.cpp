// Host build of the dual-number header and the BAL edge functor (plain C++,
// no CUDA), driven by tests/test_jet_host.py.
//
//   jet_host_check closed   chain-rule identities of mba::Jet against
//                           hand-derived closed-form gradients; exit 0 if all hold
//   jet_host_check bal      reads lines "c0..c8 X0 X1 X2" from stdin and prints,
//                           per line, for each pass width K in {12, 5, 3, 1}:
//                           pixel[2] Jc[18] Jp[6] from mba::jet_jacobian
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string_view>

#include "mba_jet.cuh"
#include "edge_bal.cuh"

using mba::Jet;

namespace {

// f(x, y) = sin(x) y / sqrt(x^2 + y^2) + cos(x y) - 3 / (x + 2) - (x - y)(y - 1)
template <class S>
S f(const S &x, const S &y) {
    using R = typename mba::scalar_of<S>::type;
    const S r = mba::ad_sqrt(x * x + y * y);
    return mba::ad_sin(x) * y / r + mba::ad_cos(x * y) - R(3) / (x + R(2)) - (x - y) * (y - R(1));
}

void grad_closed(double x, double y, double *gx, double *gy) {
    const double r = std::sqrt(x * x + y * y), r3 = r * r * r;
    *gx = std::cos(x) * y / r - std::sin(x) * y * x / r3 - std::sin(x * y) * y + 3.0 / ((x + 2.0) * (x + 2.0)) -
          (y - 1.0);
    *gy = std::sin(x) / r - std::sin(x) * y * y / r3 - std::sin(x * y) * x + (y - 1.0) - (x - y);
}

bool close(double a, double b, double tol) { return std::fabs(a - b) <= tol * (1.0 + std::fabs(b)); }

int closed() {
    const double pts[][2] = {{0.3, -1.7}, {2.5, 0.4}, {-1.1, 3.3}, {1e-3, 0.9}, {-0.7, -0.2}};
    int bad = 0;
    for (const auto &p : pts) {
        const Jet<double, 2> x(p[0], 0), y(p[1], 1);
        const Jet<double, 2> v = f(x, y);
        double gx, gy;
        grad_closed(p[0], p[1], &gx, &gy);
        if (!close(v.a, f(p[0], p[1]), 1e-15) || !close(v.v[0], gx, 1e-13) || !close(v.v[1], gy, 1e-13)) {
            std::printf("mismatch at (%g, %g): value %.17g/%.17g dx %.17g/%.17g dy %.17g/%.17g\n", p[0], p[1], v.a,
                        f(p[0], p[1]), v.v[0], gx, v.v[1], gy);
            ++bad;
        }
        // a direction outside [0, N) seeds a constant; two single-direction jets
        // give the same partials as one two-direction jet
        const Jet<double, 1> x1(p[0], 0), y1(p[1], 7), x2(p[0], -1), y2(p[1], 0);
        const Jet<double, 1> a = f(x1, y1), b = f(x2, y2);
        if (a.v[0] != v.v[0] || b.v[0] != v.v[1]) {
            std::printf("split directions differ at (%g, %g)\n", p[0], p[1]);
            ++bad;
        }
    }
    // sincos of a jet: d sin = cos dx, d cos = -sin dx, s^2 + c^2 = 1
    const Jet<double, 1> t(0.8, 0);
    Jet<double, 1> s, c;
    mba::ad_sincos(t, &s, &c);
    if (!close(s.v[0], std::cos(0.8), 1e-15) || !close(c.v[0], -std::sin(0.8), 1e-15)) ++bad;
    const Jet<double, 1> one = s * s + c * c;
    if (!close(one.a, 1.0, 1e-15) || std::fabs(one.v[0]) > 1e-15) ++bad;
    // float instantiation agrees with double to float rounding
    const Jet<float, 2> xf(0.3f, 0), yf(-1.7f, 1);
    const Jet<float, 2> vf = f(xf, yf);
    double gx, gy;
    grad_closed(0.3, -1.7, &gx, &gy);
    if (!close(vf.v[0], gx, 1e-5) || !close(vf.v[1], gy, 1e-5)) ++bad;
    if (bad) return 1;
    std::printf("closed ok\n");
    return 0;
}

template <int K>
void bal_one(const double *c, const double *X) {
    double pix[2], Jc[18], Jp[6];
    mba::jet_jacobian<K, true, true>(mba::BalEdge{}, c, X, pix, Jc, Jp);
    std::printf("%.17g %.17g", pix[0], pix[1]);
    for (double v : Jc) std::printf(" %.17g", v);
    for (double v : Jp) std::printf(" %.17g", v);
}

int bal() {
    double in[12];
    while (true) {
        for (int i = 0; i < 12; ++i)
            if (std::scanf("%lf", &in[i]) != 1) return 0;
        bal_one<12>(in, in + 9);
        std::printf(" ");
        bal_one<5>(in, in + 9);
        std::printf(" ");
        bal_one<3>(in, in + 9);
        std::printf(" ");
        bal_one<1>(in, in + 9);
        std::printf("\n");
    }
}

}  // namespace

int main(int argc, char **argv) {
    if (argc > 1 && std::string_view(argv[1]) == "closed") return closed();
    if (argc > 1 && std::string_view(argv[1]) == "bal") return bal();
    std::fprintf(stderr, "usage: jet_host_check closed|bal\n");
    return 2;
}
