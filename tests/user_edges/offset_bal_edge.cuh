// A user edge type for the build-time edge plug-in (tests/test_gpu_user_edge.py):
// the BAL camera with a principal point, pixel = BAL(c, X) + (cx, cy).  A
// problem with this edge and observations shifted by (cx, cy) is the BAL
// problem with the unshifted observations, which the oracle solves.
#pragma once

struct OffsetBalEdge {
    static constexpr int kCam = 9, kPt = 3, kOut = 2;
    static constexpr double cx = 320.0, cy = 240.0;

    template <class S>
    MBA_HD void operator()(const S *c, const S *X, S *pix) const {
        using R = typename mba::scalar_of<S>::type;
        mba::BalEdge{}(c, X, pix);
        pix[0] = pix[0] + R(cx);
        pix[1] = pix[1] + R(cy);
    }
};
