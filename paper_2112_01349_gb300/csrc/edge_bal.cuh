// edge_bal.cuh -- the BAL reprojection edge as a functor over a generic scalar,
// for the forward-mode (dual-number) Jacobian path.
//
// Camera block c = (w[3] angle-axis, t[3], f, k1, k2), point block X[3]:
//   P = R(w) X + t          (Rodrigues; first-order X + w x X + t for |w|^2 <= eps)
//   p = -(P_x, P_y) / P_z
//   pixel = f (1 + k1 |p|^2 + k2 |p|^4) p
// This is the same model as the analytic kernels (Eq. 1's residual with the
// Bundle-Adjustment-in-the-Large camera), written only as a value: its
// Jacobians come from evaluating it on mba::Jet.
#pragma once

#include <cfloat>

#include "../../include/mba_jet.cuh"

namespace mba {

template <class S>
struct scalar_of {
    using type = S;
};
template <typename T, int N>
struct scalar_of<Jet<T, N>> {
    using type = T;
};

struct BalEdge {
    static constexpr int kCam = 9, kPt = 3, kOut = 2;

    template <class S>
    MBA_HD void operator()(const S *c, const S *X, S *pix) const {
        using R = typename scalar_of<S>::type;
        const S th2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        S P0, P1, P2;
        if (value_of(th2) > R(DBL_EPSILON)) {
            const S th = ad_sqrt(th2);
            S sn, cs;
            ad_sincos(th, &sn, &cs);
            const S ith = R(1) / th;
            const S k0 = c[0] * ith, k1 = c[1] * ith, k2 = c[2] * ith;
            // X cos + (k x X) sin + k (k . X)(1 - cos)
            const S kd = (k0 * X[0] + k1 * X[1] + k2 * X[2]) * (R(1) - cs);
            P0 = X[0] * cs + (k1 * X[2] - k2 * X[1]) * sn + k0 * kd;
            P1 = X[1] * cs + (k2 * X[0] - k0 * X[2]) * sn + k1 * kd;
            P2 = X[2] * cs + (k0 * X[1] - k1 * X[0]) * sn + k2 * kd;
        } else {
            P0 = X[0] + (c[1] * X[2] - c[2] * X[1]);
            P1 = X[1] + (c[2] * X[0] - c[0] * X[2]);
            P2 = X[2] + (c[0] * X[1] - c[1] * X[0]);
        }
        P0 = P0 + c[3];
        P1 = P1 + c[4];
        P2 = P2 + c[5];
        const S iz = R(-1) / P2;
        const S px = P0 * iz, py = P1 * iz;
        const S r2 = px * px + py * py;
        const S fd = c[6] * (R(1) + r2 * (c[7] + c[8] * r2));
        pix[0] = fd * px;
        pix[1] = fd * py;
    }
};

}  // namespace mba

// A user edge type replaces BalEdge in every dual-number path when the library
// is compiled with -DMBA_EDGE_HEADER="path/to/edge.cuh" -DMBA_EDGE_TYPE=Name
// (_build.build(edge=(path, Name))): the graph's edges are then the user's
// functor, with the same interface as BalEdge (a 9-parameter camera block, a
// 3-parameter point block, a 2-vector prediction subtracted from the
// observation, and a templated operator() that also runs on mba::Jet).  The
// analytic kernels (the "-m" form, the factored FP32 product, batched windows
// and the allocation-free cost) are the BAL camera's own derivation, so such a
// library accepts MBA_JACOBIAN_AUTODIFF problems only.
#ifdef MBA_EDGE_HEADER
#include MBA_EDGE_HEADER
#endif
#ifndef MBA_EDGE_TYPE
#define MBA_EDGE_TYPE ::mba::BalEdge
#define MBA_USER_EDGE 0
#else
#define MBA_USER_EDGE 1
#endif
#define MBA_STR2(x) #x
#define MBA_STR(x) MBA_STR2(x)

namespace mba {
using Edge = MBA_EDGE_TYPE;
static_assert(Edge::kCam == 9 && Edge::kPt == 3 && Edge::kOut == 2,
              "an edge type has a 9-parameter camera, a 3-parameter point and a 2-vector residual");
constexpr bool kUserEdge = MBA_USER_EDGE != 0;
}  // namespace mba
