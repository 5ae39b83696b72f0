/*
 * ba_oracle.c -- plain, slow, obviously-correct FP64 CPU restatement of one
 * Levenberg-Marquardt iteration of BAL bundle adjustment as the MegBA paper
 * (arXiv 2112.01349) describes it.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code, header, table or helper with
 * the CUDA library and never calls it.
 *
 * What follows each passage of the paper:
 *   - objective and normal equations: Sec. 3, Eq. (1) and the H/g definitions
 *     below it (H = J^T Sigma J [+ lambda I], g = -J^T Sigma r), Sigma = I
 *     (Sec. 4.1, "assuming identity information matrix");
 *   - Schur complement blocks B, E, C, v, w: Sec. 3, Eq. (2);
 *   - reduced camera system and point back-substitution: Eqs. (3) and (4);
 *   - Hessian and gradient built per edge and summed: Sec. 4.1, Alg. 1
 *     (residual/Jacobian step, linear-system step);
 *   - PCG on the reduced camera system with block-Jacobi preconditioner B^-1:
 *     Alg. 2 (its index typos read as the textbook PCG recurrences);
 *   - implicit Schur product a = E^T x, b = C^-1 a, c = E b, d = B x, d - c:
 *     Alg. 3;
 *   - additive state update x <- x + dx: Alg. 1;
 *   - LM with a Ceres-style trust region: supplement, "Experimental Results".
 * Readings where the paper is silent (camera model, loss, damping matrix,
 * radius rule, stopping rules) are stated at each function.
 *
 * Every sum runs in a fixed order (observations of a camera or point in
 * increasing original index), so results do not depend on the OpenMP thread
 * count.  Parity for trajectory-level results (a whole LM solve) is pinned by
 * the invariant tests only; the paper prints no worked example.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_NOT_SPD 3

/* ------------------------------------------------------------------------ */
/* small dense helpers (row-major)                                            */
/* ------------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* [a]_x, the matrix with [a]_x b = a x b */
static void skew3(const double *a, double *S) {
    S[0] = 0.0;   S[1] = -a[2]; S[2] = a[1];
    S[3] = a[2];  S[4] = 0.0;   S[5] = -a[0];
    S[6] = -a[1]; S[7] = a[0];  S[8] = 0.0;
}

/* C (m x p) = A (m x q) * B (q x p) */
static void matmul(const double *A, const double *B, double *C, int m, int q, int p) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < p; ++j) {
            double s = 0.0;
            for (int k = 0; k < q; ++k) s += A[i * q + k] * B[k * p + j];
            C[i * p + j] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* BAL camera model.  The paper evaluates on BAL but never writes the model   */
/* down; this is the BAL convention: c = (w angle-axis, t, f, k1, k2),       */
/* P = R(w) X + t (Rodrigues), p = -(Px, Py)/Pz, d = 1 + k1 |p|^2 + k2 |p|^4, */
/* pixel = f d p, residual e = pixel - observation.                           */
/* ------------------------------------------------------------------------ */

/* Rotation matrix R(w) = cos(th) I + sin(th) [k]_x + (1 - cos(th)) k k^T with
 * k = w/th, or I + [w]_x when th^2 <= DBL_EPSILON (first-order form). */
static void rotation_matrix(const double *w, double *R, int *small) {
    double th2 = dot3(w, w);
    if (th2 > DBL_EPSILON) {
        double th = sqrt(th2), c = cos(th), s = sin(th);
        double k[3] = {w[0] / th, w[1] / th, w[2] / th};
        double K[9];
        skew3(k, K);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                R[i * 3 + j] = (i == j ? c : 0.0) + s * K[i * 3 + j] + (1.0 - c) * k[i] * k[j];
        *small = 0;
    } else {
        double W[9];
        skew3(w, W);
        for (int i = 0; i < 9; ++i) R[i] = W[i] + ((i % 4) == 0 ? 1.0 : 0.0);
        *small = 1;
    }
}

/* Camera-frame point: P = X cos(th) + (k x X) sin(th) + k (k.X)(1 - cos(th)) + t,
 * or X + w x X + t for th^2 <= DBL_EPSILON. */
static void camera_point(const double *cam, const double *X, double *P) {
    const double *w = cam;
    double th2 = dot3(w, w);
    if (th2 > DBL_EPSILON) {
        double th = sqrt(th2), c = cos(th), s = sin(th);
        double k[3] = {w[0] / th, w[1] / th, w[2] / th};
        double kx[3];
        cross3(k, X, kx);
        double kd = dot3(k, X) * (1.0 - c);
        for (int i = 0; i < 3; ++i) P[i] = X[i] * c + kx[i] * s + k[i] * kd + cam[3 + i];
    } else {
        double wx[3];
        cross3(w, X, wx);
        for (int i = 0; i < 3; ++i) P[i] = X[i] + wx[i] + cam[3 + i];
    }
}

void orc_project(const double *cam, const double *X, double *pix) {
    double P[3];
    camera_point(cam, X, P);
    double px = -P[0] / P[2], py = -P[1] / P[2];
    double r2 = px * px + py * py;
    double d = 1.0 + cam[7] * r2 + cam[8] * r2 * r2;
    pix[0] = cam[6] * d * px;
    pix[1] = cam[6] * d * py;
}

/* Residual and analytic Jacobian by the chain rule.  Jc is 2x9 (w, t, f, k1,
 * k2), Jp is 2x3, both row-major.  dP/dw = -R [X]_x (w w^T + (R^T - I)[w]_x)/th^2
 * (Gallego & Yezzi, J. Math. Imaging Vis. 2015); first-order branch -[X]_x. */
void orc_residual_jacobian(const double *cam, const double *X, const double *u, double *e,
                           double *Jc, double *Jp) {
    const double *w = cam;
    double R[9];
    int small;
    rotation_matrix(w, R, &small);
    double P[3];
    camera_point(cam, X, P);

    double dPdw[9];
    double Xs[9];
    skew3(X, Xs);
    if (!small) {
        double th2 = dot3(w, w);
        double Ws[9], RtI[9], M[9], T1[9];
        skew3(w, Ws);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) RtI[i * 3 + j] = R[j * 3 + i] - (i == j ? 1.0 : 0.0);
        matmul(RtI, Ws, M, 3, 3, 3);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i * 3 + j] = (M[i * 3 + j] + w[i] * w[j]) / th2;
        matmul(R, Xs, T1, 3, 3, 3);
        matmul(T1, M, dPdw, 3, 3, 3);
        for (int i = 0; i < 9; ++i) dPdw[i] = -dPdw[i];
    } else {
        for (int i = 0; i < 9; ++i) dPdw[i] = -Xs[i];
    }

    double iz = 1.0 / P[2];
    double px = -P[0] * iz, py = -P[1] * iz;
    double dpdP[6] = {-iz, 0.0, P[0] * iz * iz, 0.0, -iz, P[1] * iz * iz};
    double f = cam[6], k1 = cam[7], k2 = cam[8];
    double r2 = px * px + py * py;
    double d = 1.0 + k1 * r2 + k2 * r2 * r2;
    double dd = 2.0 * k1 + 4.0 * k2 * r2; /* d(d)/dp = dd * p */
    double dpix_dp[4] = {f * (d + dd * px * px), f * dd * px * py, f * dd * py * px, f * (d + dd * py * py)};
    double dpix_dP[6];
    matmul(dpix_dp, dpdP, dpix_dP, 2, 2, 3);

    e[0] = f * d * px - u[0];
    e[1] = f * d * py - u[1];

    double Jw[6];
    matmul(dpix_dP, dPdw, Jw, 2, 3, 3);
    for (int r = 0; r < 2; ++r) {
        double pr = r == 0 ? px : py;
        Jc[r * 9 + 0] = Jw[r * 3 + 0];
        Jc[r * 9 + 1] = Jw[r * 3 + 1];
        Jc[r * 9 + 2] = Jw[r * 3 + 2];
        Jc[r * 9 + 3] = dpix_dP[r * 3 + 0];
        Jc[r * 9 + 4] = dpix_dP[r * 3 + 1];
        Jc[r * 9 + 5] = dpix_dP[r * 3 + 2];
        Jc[r * 9 + 6] = d * pr;
        Jc[r * 9 + 7] = f * r2 * pr;
        Jc[r * 9 + 8] = f * r2 * r2 * pr;
    }
    /* dP/dX = R (I + [w]_x in the first-order branch, which rotation_matrix returns) */
    matmul(dpix_dP, R, Jp, 2, 3, 3);
}

/* Loss on the squared residual norm s.  Plain: rho(s) = s, weight 1.  Huber
 * with threshold delta (pixels): rho(s) = s for s <= delta^2, else
 * 2 delta sqrt(s) - delta^2; the IRLS weight is rho'(s) (1 or delta/sqrt(s)). */
static void loss_eval(int loss, double delta, double s, double *rho, double *weight) {
    if (loss == 1 && s > delta * delta) {
        double r = sqrt(s);
        *rho = 2.0 * delta * r - delta * delta;
        *weight = delta / r;
    } else {
        *rho = s;
        *weight = 1.0;
    }
}

void orc_loss(int loss, double delta, double s, double *rho, double *weight) { loss_eval(loss, delta, s, rho, weight); }

/* Cost F = 1/2 sum_k rho(|e_k|^2) (Eq. 1 with Sigma = I), plus optional
 * per-observation e (n*2), Jc (n*18), Jp (n*6) and weights (n), input order. */
int orc_evaluate(int32_t nc, int32_t np, int64_t n, const double *cams, const double *pts,
                 const double *obs, const int32_t *cam_idx, const int32_t *pt_idx, int loss,
                 double delta, double *cost, double *e_out, double *jc_out, double *jp_out,
                 double *w_out) {
    if (n < 1 || nc < 1 || np < 1) return ORC_ERR_ARG;
    double *rho = (double *)malloc(sizeof(double) * (size_t)n);
    if (!rho) return ORC_ERR_OOM;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double e[2], Jc[18], Jp[6], r, wt;
        orc_residual_jacobian(cams + 9 * (int64_t)cam_idx[k], pts + 3 * (int64_t)pt_idx[k], obs + 2 * k, e, Jc, Jp);
        loss_eval(loss, delta, e[0] * e[0] + e[1] * e[1], &r, &wt);
        rho[k] = r;
        if (e_out) { e_out[2 * k] = e[0]; e_out[2 * k + 1] = e[1]; }
        if (jc_out) memcpy(jc_out + 18 * k, Jc, sizeof(Jc));
        if (jp_out) memcpy(jp_out + 6 * k, Jp, sizeof(Jp));
        if (w_out) w_out[k] = wt;
    }
    double F = 0.0;
    for (int64_t k = 0; k < n; ++k) F += rho[k];
    *cost = 0.5 * F;
    free(rho);
    return ORC_OK;
}

/* Cost only, from the residual alone (no Jacobian). */
static double cost_only(int64_t n, const double *cams, const double *pts, const double *obs,
                        const int32_t *cam_idx, const int32_t *pt_idx, int loss, double delta,
                        double *scratch) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double pix[2], r, wt;
        orc_project(cams + 9 * (int64_t)cam_idx[k], pts + 3 * (int64_t)pt_idx[k], pix);
        double ex = pix[0] - obs[2 * k], ey = pix[1] - obs[2 * k + 1];
        loss_eval(loss, delta, ex * ex + ey * ey, &r, &wt);
        scratch[k] = r;
    }
    double F = 0.0;
    for (int64_t k = 0; k < n; ++k) F += scratch[k];
    return 0.5 * F;
}

/* ------------------------------------------------------------------------ */
/* Stable counting sort: perm lists observation indices grouped by key in     */
/* increasing key order, original order inside a key; ptr is the CSR offset   */
/* array (nkeys + 1).  This is the CSR layout of E / E^T (Sec. 4.1).          */
/* ------------------------------------------------------------------------ */
int orc_stable_sort(int64_t n, const int32_t *keys, int32_t nkeys, int32_t *perm, int32_t *ptr) {
    for (int32_t k = 0; k <= nkeys; ++k) ptr[k] = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (keys[k] < 0 || keys[k] >= nkeys) return ORC_ERR_ARG;
        ptr[keys[k] + 1]++;
    }
    for (int32_t k = 0; k < nkeys; ++k) ptr[k + 1] += ptr[k];
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nkeys > 0 ? nkeys : 1));
    if (!next) return ORC_ERR_OOM;
    for (int32_t k = 0; k < nkeys; ++k) next[k] = ptr[k];
    for (int64_t k = 0; k < n; ++k) perm[next[keys[k]]++] = (int32_t)k;
    free(next);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Linearisation (Alg. 1, residual/Jacobian and linear-system steps).         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t nc, np;
    int64_t n;
    const int32_t *cam_idx, *pt_idx;
    int32_t *cam_perm, *cam_ptr; /* observations of camera i: cam_perm[cam_ptr[i] .. cam_ptr[i+1]) */
    int32_t *pt_perm, *pt_ptr;   /* observations of point j */
    double *e, *W;               /* n*2, n */
    double *Jc, *Jp;             /* n*18, n*6 */
    double *E;                   /* n*27: E_k = W_k Jc_k^T Jp_k (9x3), the non-zero block of E */
    double *Hpp, *v;             /* nc*81, nc*9 : B block and camera gradient */
    double *Hll, *w;             /* np*9,  np*3 : C block and point gradient */
    const uint8_t *cam_fixed;    /* nc or NULL: nonzero = camera held constant */
    const uint8_t *pt_fixed;     /* np or NULL: nonzero = point held constant */
} lin_t;

static void lin_free(lin_t *L) {
    free(L->cam_perm); free(L->cam_ptr); free(L->pt_perm); free(L->pt_ptr);
    free(L->e); free(L->W); free(L->Jc); free(L->Jp); free(L->E);
    free(L->Hpp); free(L->v); free(L->Hll); free(L->w);
    memset(L, 0, sizeof(*L));
}

static int lin_alloc(lin_t *L, int32_t nc, int32_t np, int64_t n, const int32_t *cam_idx, const int32_t *pt_idx) {
    memset(L, 0, sizeof(*L));
    L->nc = nc; L->np = np; L->n = n; L->cam_idx = cam_idx; L->pt_idx = pt_idx;
    L->cam_perm = malloc(sizeof(int32_t) * n); L->cam_ptr = malloc(sizeof(int32_t) * (nc + 1));
    L->pt_perm = malloc(sizeof(int32_t) * n);  L->pt_ptr = malloc(sizeof(int32_t) * (np + 1));
    L->e = malloc(sizeof(double) * 2 * n); L->W = malloc(sizeof(double) * n);
    L->Jc = malloc(sizeof(double) * 18 * n); L->Jp = malloc(sizeof(double) * 6 * n);
    L->E = malloc(sizeof(double) * 27 * n);
    L->Hpp = malloc(sizeof(double) * 81 * nc); L->v = malloc(sizeof(double) * 9 * nc);
    L->Hll = malloc(sizeof(double) * 9 * np);  L->w = malloc(sizeof(double) * 3 * np);
    if (!L->cam_perm || !L->cam_ptr || !L->pt_perm || !L->pt_ptr || !L->e || !L->W || !L->Jc ||
        !L->Jp || !L->E || !L->Hpp || !L->v || !L->Hll || !L->w) {
        lin_free(L);
        return ORC_ERR_OOM;
    }
    if (orc_stable_sort(n, cam_idx, nc, L->cam_perm, L->cam_ptr) != ORC_OK) { lin_free(L); return ORC_ERR_ARG; }
    if (orc_stable_sort(n, pt_idx, np, L->pt_perm, L->pt_ptr) != ORC_OK) { lin_free(L); return ORC_ERR_ARG; }
    return ORC_OK;
}

/* r_k, J_k at the current state; then [B E; E^T C] = J^T W J and [v w] = -J^T W r
 * as sums of per-edge terms (Alg. 1).  W_k is the IRLS weight rho'(s_k).
 * Fixed nodes (nodes held constant, the g2o / Ceres convention the paper's
 * graph API follows, Sec. 5.3): the Jacobian columns of a fixed camera or
 * point are zero.  Their rows of B, C, E and the gradient vanish, the damping
 * floor keeps their damped blocks positive definite, and the damped step is
 * that of the problem over the free parameters alone, zero on the fixed ones. */
static void linearise(lin_t *L, const double *cams, const double *pts, const double *obs, int loss, double delta) {
    const int64_t n = L->n;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double *e = L->e + 2 * k, *Jc = L->Jc + 18 * k, *Jp = L->Jp + 6 * k, *E = L->E + 27 * k;
        orc_residual_jacobian(cams + 9 * (int64_t)L->cam_idx[k], pts + 3 * (int64_t)L->pt_idx[k], obs + 2 * k, e, Jc, Jp);
        if (L->cam_fixed && L->cam_fixed[L->cam_idx[k]]) memset(Jc, 0, sizeof(double) * 18);
        if (L->pt_fixed && L->pt_fixed[L->pt_idx[k]]) memset(Jp, 0, sizeof(double) * 6);
        double rho, wt;
        loss_eval(loss, delta, e[0] * e[0] + e[1] * e[1], &rho, &wt);
        L->W[k] = wt;
        for (int a = 0; a < 9; ++a)
            for (int b = 0; b < 3; ++b) E[a * 3 + b] = wt * (Jc[a] * Jp[b] + Jc[9 + a] * Jp[3 + b]);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t i = 0; i < L->nc; ++i) {
        double *H = L->Hpp + 81 * (int64_t)i, *v = L->v + 9 * (int64_t)i;
        memset(H, 0, sizeof(double) * 81);
        memset(v, 0, sizeof(double) * 9);
        for (int32_t s = L->cam_ptr[i]; s < L->cam_ptr[i + 1]; ++s) {
            int64_t k = L->cam_perm[s];
            const double *Jc = L->Jc + 18 * k, *e = L->e + 2 * k;
            double wt = L->W[k];
            for (int a = 0; a < 9; ++a) {
                for (int b = 0; b < 9; ++b) H[a * 9 + b] += wt * (Jc[a] * Jc[b] + Jc[9 + a] * Jc[9 + b]);
                v[a] -= wt * (Jc[a] * e[0] + Jc[9 + a] * e[1]);
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < L->np; ++j) {
        double *H = L->Hll + 9 * (int64_t)j, *w = L->w + 3 * (int64_t)j;
        memset(H, 0, sizeof(double) * 9);
        memset(w, 0, sizeof(double) * 3);
        for (int32_t s = L->pt_ptr[j]; s < L->pt_ptr[j + 1]; ++s) {
            int64_t k = L->pt_perm[s];
            const double *Jp = L->Jp + 6 * k, *e = L->e + 2 * k;
            double wt = L->W[k];
            for (int a = 0; a < 3; ++a) {
                for (int b = 0; b < 3; ++b) H[a * 3 + b] += wt * (Jp[a] * Jp[b] + Jp[3 + a] * Jp[3 + b]);
                w[a] -= wt * (Jp[a] * e[0] + Jp[3 + a] * e[1]);
            }
        }
    }
}

/* Blocks B (nc*81), v (nc*9), C (np*9), w (np*3) and optionally E (n*27). */
int orc_blocks(int32_t nc, int32_t np, int64_t n, const double *cams, const double *pts, const double *obs,
               const int32_t *cam_idx, const int32_t *pt_idx, int loss, double delta, double *Hpp, double *v,
               double *Hll, double *w, double *E) {
    lin_t L;
    int rc = lin_alloc(&L, nc, np, n, cam_idx, pt_idx);
    if (rc) return rc;
    linearise(&L, cams, pts, obs, loss, delta);
    memcpy(Hpp, L.Hpp, sizeof(double) * 81 * nc);
    memcpy(v, L.v, sizeof(double) * 9 * nc);
    memcpy(Hll, L.Hll, sizeof(double) * 9 * np);
    memcpy(w, L.w, sizeof(double) * 3 * np);
    if (E) memcpy(E, L.E, sizeof(double) * 27 * n);
    lin_free(&L);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Damping.  The paper writes H + lambda I (Sec. 3) but also says its LM uses */
/* the Ceres trust-region strategy (supplement).  Reading: damping mode 0     */
/* adds mu * clamp(diag(H), 1e-6, 1e32) (the Ceres form, default); mode 1     */
/* adds mu * I (the literal form).  Applied to B and C before elimination.    */
/* ------------------------------------------------------------------------ */
static double damp_term(int damping, double diag_entry) {
    if (damping == 1) return 1.0;
    double d = diag_entry;
    if (d < 1e-6) d = 1e-6;
    if (d > 1e32) d = 1e32;
    return d;
}

typedef struct {
    double *Bd;   /* nc*81: damped camera blocks B~ */
    double *Lb;   /* nc*81: Cholesky factor of B~ (lower, row-major) */
    double *Cinv; /* np*9: inverse of damped point blocks C~ */
} damped_t;

static void damped_free(damped_t *D) { free(D->Bd); free(D->Lb); free(D->Cinv); memset(D, 0, sizeof(*D)); }

/* In-place lower Cholesky of an m x m SPD matrix (row-major).  Returns 0 if
 * a pivot is not positive. */
static int cholesky(double *A, int m) {
    for (int j = 0; j < m; ++j) {
        double s = A[j * m + j];
        for (int k = 0; k < j; ++k) s -= A[j * m + k] * A[j * m + k];
        if (!(s > 0.0)) return 0;
        double ljj = sqrt(s);
        A[j * m + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            double t = A[i * m + j];
            for (int k = 0; k < j; ++k) t -= A[i * m + k] * A[j * m + k];
            A[i * m + j] = t / ljj;
        }
        for (int i = 0; i < j; ++i) A[i * m + j] = 0.0;
    }
    return 1;
}

/* Solve (L L^T) x = b for one m x m factor. */
static void chol_solve(const double *Lf, int m, const double *b, double *x) {
    double y[16];
    for (int i = 0; i < m; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= Lf[i * m + k] * y[k];
        y[i] = s / Lf[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < m; ++k) s -= Lf[k * m + i] * x[k];
        x[i] = s / Lf[i * m + i];
    }
}

/* 3x3 inverse by the adjugate. */
static int inverse3(const double *A, double *Ai) {
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(det != 0.0) || !isfinite(det)) return 0;
    double id = 1.0 / det;
    Ai[0] = c00 * id;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    Ai[3] = c01 * id;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    Ai[6] = c02 * id;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return 1;
}

static int damp(const lin_t *L, double mu, int damping, damped_t *D) {
    D->Bd = malloc(sizeof(double) * 81 * L->nc);
    D->Lb = malloc(sizeof(double) * 81 * L->nc);
    D->Cinv = malloc(sizeof(double) * 9 * L->np);
    if (!D->Bd || !D->Lb || !D->Cinv) { damped_free(D); return ORC_ERR_OOM; }
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int32_t i = 0; i < L->nc; ++i) {
        double *B = D->Bd + 81 * (int64_t)i, *Lf = D->Lb + 81 * (int64_t)i;
        memcpy(B, L->Hpp + 81 * (int64_t)i, sizeof(double) * 81);
        for (int a = 0; a < 9; ++a) B[a * 9 + a] += mu * damp_term(damping, B[a * 9 + a]);
        memcpy(Lf, B, sizeof(double) * 81);
        if (!cholesky(Lf, 9)) bad |= 1;
    }
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int32_t j = 0; j < L->np; ++j) {
        double C[9];
        memcpy(C, L->Hll + 9 * (int64_t)j, sizeof(C));
        for (int a = 0; a < 3; ++a) C[a * 3 + a] += mu * damp_term(damping, C[a * 3 + a]);
        if (!inverse3(C, D->Cinv + 9 * (int64_t)j)) bad |= 1;
    }
    if (bad) { damped_free(D); return ORC_ERR_NOT_SPD; }
    return ORC_OK;
}

/* Schur-Jacobi preconditioner (a solver variant beside Alg. 2's block-Jacobi
 * on B~): the camera blocks S~_ii = B~_i - sum_k E_k C~_j(k)^-1 E_k^T over the
 * observations k of camera i.  When every (camera, point) pair is observed at
 * most once these are exactly the diagonal blocks of S = B~ - E C~^-1 E^T (Eq. 3).
 * Their Cholesky factors replace those of B~ in D->Lb; a block that is not
 * positive definite keeps the factor of B~_i.  Blocks are written to Sjd
 * (nc*81) if it is not NULL. */
static void schur_jacobi(const lin_t *L, damped_t *D, double *Sjd) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t i = 0; i < L->nc; ++i) {
        double S[81];
        memcpy(S, D->Bd + 81 * (int64_t)i, sizeof(S));
        for (int32_t s = L->cam_ptr[i]; s < L->cam_ptr[i + 1]; ++s) {
            const int64_t k = L->cam_perm[s];
            const double *Ek = L->E + 27 * k, *Ci = D->Cinv + 9 * (int64_t)L->pt_idx[k];
            double EC[27];
            matmul(Ek, Ci, EC, 9, 3, 3);
            for (int a = 0; a < 9; ++a)
                for (int b = 0; b < 9; ++b)
                    S[a * 9 + b] -= EC[a * 3] * Ek[b * 3] + EC[a * 3 + 1] * Ek[b * 3 + 1] + EC[a * 3 + 2] * Ek[b * 3 + 2];
        }
        if (Sjd) memcpy(Sjd + 81 * (int64_t)i, S, sizeof(S));
        double F[81];
        memcpy(F, S, sizeof(F));
        if (cholesky(F, 9)) memcpy(D->Lb + 81 * (int64_t)i, F, sizeof(F));
    }
}

/* ------------------------------------------------------------------------ */
/* Schur elimination (Eqs. 3, 4; Alg. 3).                                    */
/* ------------------------------------------------------------------------ */

/* y = S x with S = B~ - E C~^-1 E^T, computed without forming S (Alg. 3):
 * a = E^T x, b = C~^-1 a, c = E b, d = B~ x, y = d - c.  Scratch: a, b (np*3). */
static void schur_matvec(const lin_t *L, const damped_t *D, const double *x, double *y, double *a, double *b) {
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < L->np; ++j) {
        double aj[3] = {0.0, 0.0, 0.0};
        for (int32_t s = L->pt_ptr[j]; s < L->pt_ptr[j + 1]; ++s) {
            int64_t k = L->pt_perm[s];
            const double *E = L->E + 27 * k, *xi = x + 9 * (int64_t)L->cam_idx[k];
            for (int c = 0; c < 3; ++c)
                for (int r = 0; r < 9; ++r) aj[c] += E[r * 3 + c] * xi[r];
        }
        const double *Ci = D->Cinv + 9 * (int64_t)j;
        for (int r = 0; r < 3; ++r) {
            a[3 * (int64_t)j + r] = aj[r];
            b[3 * (int64_t)j + r] = Ci[r * 3] * aj[0] + Ci[r * 3 + 1] * aj[1] + Ci[r * 3 + 2] * aj[2];
        }
    }
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < L->nc; ++i) {
        double c[9] = {0};
        for (int32_t s = L->cam_ptr[i]; s < L->cam_ptr[i + 1]; ++s) {
            int64_t k = L->cam_perm[s];
            const double *E = L->E + 27 * k, *bj = b + 3 * (int64_t)L->pt_idx[k];
            for (int r = 0; r < 9; ++r) c[r] += E[r * 3] * bj[0] + E[r * 3 + 1] * bj[1] + E[r * 3 + 2] * bj[2];
        }
        const double *B = D->Bd + 81 * (int64_t)i, *xi = x + 9 * (int64_t)i;
        for (int r = 0; r < 9; ++r) {
            double d = 0.0;
            for (int q = 0; q < 9; ++q) d += B[r * 9 + q] * xi[q];
            y[9 * (int64_t)i + r] = d - c[r];
        }
    }
}

/* Reduced-camera right-hand side v - E C~^-1 w (Eq. 3; Alg. 1 alpha/g steps). */
static void schur_rhs(const lin_t *L, const damped_t *D, double *g, double *b) {
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < L->np; ++j) {
        const double *Ci = D->Cinv + 9 * (int64_t)j, *wj = L->w + 3 * (int64_t)j;
        for (int r = 0; r < 3; ++r) b[3 * (int64_t)j + r] = Ci[r * 3] * wj[0] + Ci[r * 3 + 1] * wj[1] + Ci[r * 3 + 2] * wj[2];
    }
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < L->nc; ++i) {
        double c[9] = {0};
        for (int32_t s = L->cam_ptr[i]; s < L->cam_ptr[i + 1]; ++s) {
            int64_t k = L->cam_perm[s];
            const double *E = L->E + 27 * k, *bj = b + 3 * (int64_t)L->pt_idx[k];
            for (int r = 0; r < 9; ++r) c[r] += E[r * 3] * bj[0] + E[r * 3 + 1] * bj[1] + E[r * 3 + 2] * bj[2];
        }
        for (int r = 0; r < 9; ++r) g[9 * (int64_t)i + r] = L->v[9 * (int64_t)i + r] - c[r];
    }
}

/* Explicit dense S (9nc x 9nc) for small problems (Eq. 3 formed literally). */
static void schur_explicit(const lin_t *L, const damped_t *D, double *S) {
    const int64_t m = 9 * (int64_t)L->nc;
    memset(S, 0, sizeof(double) * m * m);
    for (int32_t i = 0; i < L->nc; ++i)
        for (int a = 0; a < 9; ++a)
            for (int b = 0; b < 9; ++b) S[(9 * i + a) * m + 9 * i + b] = D->Bd[81 * (int64_t)i + a * 9 + b];
    for (int32_t j = 0; j < L->np; ++j) {
        const double *Ci = D->Cinv + 9 * (int64_t)j;
        for (int32_t s = L->pt_ptr[j]; s < L->pt_ptr[j + 1]; ++s) {
            int64_t k = L->pt_perm[s];
            const double *Ek = L->E + 27 * k;
            double EC[27]; /* E_k C~^-1 */
            matmul(Ek, Ci, EC, 9, 3, 3);
            for (int32_t t = L->pt_ptr[j]; t < L->pt_ptr[j + 1]; ++t) {
                int64_t l = L->pt_perm[t];
                const double *El = L->E + 27 * l;
                int64_t ri = 9 * (int64_t)L->cam_idx[k], ci = 9 * (int64_t)L->cam_idx[l];
                for (int a = 0; a < 9; ++a)
                    for (int b = 0; b < 9; ++b)
                        S[(ri + a) * m + ci + b] -= EC[a * 3] * El[b * 3] + EC[a * 3 + 1] * El[b * 3 + 1] + EC[a * 3 + 2] * El[b * 3 + 2];
            }
        }
    }
}

static double vdot(const double *a, const double *b, int64_t m) {
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
}

/* PCG on S x = g (Alg. 2).  Reading of its recurrences: x0 = 0, r0 = g;
 * each step z = M^-1 r with M = blockdiag(B~_i); rho = r.z; p = z on the first
 * step, else p = z + (rho/rho_prev) p; q = S p; alpha = rho/(p.q); x += alpha p;
 * r -= alpha q.  Stop when |r|_2 <= tol |r0|_2 or after max_iter steps; stop
 * early (keeping x) if rho is not finite or p.q is not positive.
 * S is applied implicitly (Alg. 3) or, if Sd != NULL, as the dense matrix. */
static int pcg(const lin_t *L, const damped_t *D, const double *Sd, const double *g, double *x, int max_iter,
               double tol, double *rel_res) {
    const int64_t m = 9 * (int64_t)L->nc;
    double *r = malloc(sizeof(double) * m), *z = malloc(sizeof(double) * m), *p = malloc(sizeof(double) * m),
           *q = malloc(sizeof(double) * m);
    double *sa = malloc(sizeof(double) * 3 * (size_t)L->np), *sb = malloc(sizeof(double) * 3 * (size_t)L->np);
    int n = 0;
    memset(x, 0, sizeof(double) * m);
    memcpy(r, g, sizeof(double) * m);
    double r0 = sqrt(vdot(r, r, m)), rho_prev = 0.0, rn = r0;
    if (r0 > 0.0) {
        for (;;) {
            for (int32_t i = 0; i < L->nc; ++i) chol_solve(D->Lb + 81 * (int64_t)i, 9, r + 9 * (int64_t)i, z + 9 * (int64_t)i);
            double rho = vdot(r, z, m);
            if (!isfinite(rho)) break;
            if (n == 0) memcpy(p, z, sizeof(double) * m);
            else {
                double beta = rho / rho_prev;
                for (int64_t t = 0; t < m; ++t) p[t] = z[t] + beta * p[t];
            }
            if (Sd) {
                for (int64_t a = 0; a < m; ++a) q[a] = vdot(Sd + a * m, p, m);
            } else {
                schur_matvec(L, D, p, q, sa, sb);
            }
            double pq = vdot(p, q, m);
            if (!(pq > 0.0) || !isfinite(pq)) break;
            double alpha = rho / pq;
            for (int64_t t = 0; t < m; ++t) { x[t] += alpha * p[t]; r[t] -= alpha * q[t]; }
            ++n;
            rho_prev = rho;
            rn = sqrt(vdot(r, r, m));
            if (rn <= tol * r0 || n >= max_iter) break;
        }
    }
    if (rel_res) *rel_res = r0 > 0.0 ? rn / r0 : 0.0;
    free(r); free(z); free(p); free(q); free(sa); free(sb);
    return n;
}

/* Single-reduction form of the same PCG (a solver variant, off by default):
 * A. T. Chronopoulos and C. W. Gear, "s-step iterative methods for symmetric
 * linear systems", J. Comput. Appl. Math. 25 (1989), the one-step method with
 * a preconditioner.  Each step forms u = M^-1 r and w = S u, then takes the
 * three inner products gamma = r.u, delta = w.u and r.r together, which a
 * parallel implementation gathers in one global reduction instead of two:
 *   beta  = gamma / gamma_prev               (0 on the first step)
 *   alpha = gamma / (delta - beta gamma / alpha_prev)   (gamma / delta first)
 *   p = u + beta p,  s = w + beta s          (so s = S p),
 *   x += alpha p,    r -= alpha s.
 * The denominator of alpha equals p.S p in exact arithmetic (expand p.S p with
 * p = u + beta p_prev, use r.u_prev = 0 and p_prev.S p_prev =
 * gamma_prev / alpha_prev), so the iterates are those of pcg() above; only
 * the rounding differs.  Start, stopping test and breakdown rules as there:
 * stop, keeping x, if gamma is not finite or the denominator is not positive. */
static int pcg_single_reduction(const lin_t *L, const damped_t *D, const double *Sd, const double *g, double *x,
                                int max_iter, double tol, double *rel_res) {
    const int64_t m = 9 * (int64_t)L->nc;
    double *r = malloc(sizeof(double) * m), *u = malloc(sizeof(double) * m), *w = malloc(sizeof(double) * m),
           *p = malloc(sizeof(double) * m), *sv = malloc(sizeof(double) * m);
    double *sa = malloc(sizeof(double) * 3 * (size_t)L->np), *sb = malloc(sizeof(double) * 3 * (size_t)L->np);
    int n = 0;
    memset(x, 0, sizeof(double) * m);
    memcpy(r, g, sizeof(double) * m);
    double r0 = sqrt(vdot(r, r, m)), rn = r0, gamma_prev = 0.0, alpha_prev = 0.0;
    if (r0 > 0.0) {
        for (;;) {
            for (int32_t i = 0; i < L->nc; ++i) chol_solve(D->Lb + 81 * (int64_t)i, 9, r + 9 * (int64_t)i, u + 9 * (int64_t)i);
            if (Sd) {
                for (int64_t a = 0; a < m; ++a) w[a] = vdot(Sd + a * m, u, m);
            } else {
                schur_matvec(L, D, u, w, sa, sb);
            }
            const double gamma = vdot(r, u, m), delta = vdot(w, u, m);
            if (!isfinite(gamma)) break;
            const double beta = n == 0 ? 0.0 : gamma / gamma_prev;
            const double den = n == 0 ? delta : delta - beta * gamma / alpha_prev;
            if (!(den > 0.0) || !isfinite(den)) break;
            const double alpha = gamma / den;
            for (int64_t t = 0; t < m; ++t) {
                p[t] = n == 0 ? u[t] : u[t] + beta * p[t];
                sv[t] = n == 0 ? w[t] : w[t] + beta * sv[t];
                x[t] += alpha * p[t];
                r[t] -= alpha * sv[t];
            }
            ++n;
            gamma_prev = gamma;
            alpha_prev = alpha;
            rn = sqrt(vdot(r, r, m));
            if (rn <= tol * r0 || n >= max_iter) break;
        }
    }
    if (rel_res) *rel_res = r0 > 0.0 ? rn / r0 : 0.0;
    free(r); free(u); free(w); free(p); free(sv); free(sa); free(sb);
    return n;
}

/* The PCG of a damped solve: variant 0 the two-reduction loop of Alg. 2,
 * 1 the single-reduction form. */
static int pcg_any(int variant, const lin_t *L, const damped_t *D, const double *Sd, const double *g, double *x,
                   int max_iter, double tol, double *rel_res) {
    return variant == 1 ? pcg_single_reduction(L, D, Sd, g, x, max_iter, tol, rel_res)
                        : pcg(L, D, Sd, g, x, max_iter, tol, rel_res);
}

/* Dense Cholesky solve of S x = g (small problems). */
static int dense_solve(double *S, int64_t m, const double *g, double *x) {
    for (int64_t j = 0; j < m; ++j) {
        double s = S[j * m + j];
        for (int64_t k = 0; k < j; ++k) s -= S[j * m + k] * S[j * m + k];
        if (!(s > 0.0)) return ORC_ERR_NOT_SPD;
        double l = sqrt(s);
        S[j * m + j] = l;
        for (int64_t i = j + 1; i < m; ++i) {
            double t = S[i * m + j];
            for (int64_t k = 0; k < j; ++k) t -= S[i * m + k] * S[j * m + k];
            S[i * m + j] = t / l;
        }
    }
    double *y = malloc(sizeof(double) * m);
    for (int64_t i = 0; i < m; ++i) {
        double s = g[i];
        for (int64_t k = 0; k < i; ++k) s -= S[i * m + k] * y[k];
        y[i] = s / S[i * m + i];
    }
    for (int64_t i = m - 1; i >= 0; --i) {
        double s = y[i];
        for (int64_t k = i + 1; k < m; ++k) s -= S[k * m + i] * x[k];
        x[i] = s / S[i * m + i];
    }
    free(y);
    return ORC_OK;
}

/* Point back-substitution dp_j = C~_j^-1 (w_j - sum_k E_k^T dc_i(k)) (Eq. 4). */
static void back_substitute(const lin_t *L, const damped_t *D, const double *dc, double *dp) {
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < L->np; ++j) {
        double t[3] = {L->w[3 * (int64_t)j], L->w[3 * (int64_t)j + 1], L->w[3 * (int64_t)j + 2]};
        for (int32_t s = L->pt_ptr[j]; s < L->pt_ptr[j + 1]; ++s) {
            int64_t k = L->pt_perm[s];
            const double *E = L->E + 27 * k, *xi = dc + 9 * (int64_t)L->cam_idx[k];
            for (int c = 0; c < 3; ++c)
                for (int r = 0; r < 9; ++r) t[c] -= E[r * 3 + c] * xi[r];
        }
        const double *Ci = D->Cinv + 9 * (int64_t)j;
        for (int r = 0; r < 3; ++r) dp[3 * (int64_t)j + r] = Ci[r * 3] * t[0] + Ci[r * 3 + 1] * t[1] + Ci[r * 3 + 2] * t[2];
    }
}

/* Linear model decrease 1/2 sum_k W_k (|e_k|^2 - |e_k + J_k dx|^2). */
static double model_decrease(const lin_t *L, const double *dc, const double *dp, double *scratch) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < L->n; ++k) {
        const double *Jc = L->Jc + 18 * k, *Jp = L->Jp + 6 * k, *e = L->e + 2 * k;
        const double *xc = dc + 9 * (int64_t)L->cam_idx[k], *xp = dp + 3 * (int64_t)L->pt_idx[k];
        double f[2];
        for (int r = 0; r < 2; ++r) {
            double s = e[r];
            for (int a = 0; a < 9; ++a) s += Jc[r * 9 + a] * xc[a];
            for (int a = 0; a < 3; ++a) s += Jp[r * 3 + a] * xp[a];
            f[r] = s;
        }
        scratch[k] = L->W[k] * ((e[0] * e[0] + e[1] * e[1]) - (f[0] * f[0] + f[1] * f[1]));
    }
    double s = 0.0;
    for (int64_t k = 0; k < L->n; ++k) s += scratch[k];
    return 0.5 * s;
}

/* One damped step at the current linearisation: solve (H + mu D) dx = g by
 * Schur elimination.  schur_mode: 0 = PCG with the implicit product (Alg. 2+3),
 * 1 = PCG with the explicit dense S, 2 = dense Cholesky of S. */
/* One damped solve.  precond: 0 block-Jacobi on B~ (Alg. 2), 1 Schur-Jacobi.
 * g0n != NULL turns on the inexact-Newton forcing sequence: the PCG tolerance
 * becomes max(pcg_tol, min(0.1, sqrt(|g| / |g_first|))), |g| the norm of this
 * solve's reduced right-hand side and |g_first| that of the first solve
 * (*g0n <= 0 on entry marks the first solve; it is then set). */
static int damped_step(const lin_t *L, double mu, int damping, int schur_mode, int pcg_max, double pcg_tol,
                       double *dc, double *dp, int *pcg_iters, double *rel_res, int precond, double *g0n,
                       int variant) {
    damped_t D;
    int rc = damp(L, mu, damping, &D);
    if (rc) return rc;
    if (precond == 1) schur_jacobi(L, &D, NULL);
    const int64_t m = 9 * (int64_t)L->nc;
    double *g = malloc(sizeof(double) * m), *sb = malloc(sizeof(double) * 3 * (size_t)L->np);
    schur_rhs(L, &D, g, sb);
    if (g0n) {
        const double gn = sqrt(vdot(g, g, m));
        if (!(*g0n > 0.0)) *g0n = gn;
        const double eta = *g0n > 0.0 ? sqrt(gn / *g0n) : 0.0;
        const double t = eta < 0.1 ? eta : 0.1;
        if (t > pcg_tol) pcg_tol = t;
    }
    *pcg_iters = 0;
    if (rel_res) *rel_res = 0.0;
    if (schur_mode == 0) {
        *pcg_iters = pcg_any(variant, L, &D, NULL, g, dc, pcg_max, pcg_tol, rel_res);
    } else {
        double *S = malloc(sizeof(double) * m * m);
        if (!S) { free(g); free(sb); damped_free(&D); return ORC_ERR_OOM; }
        schur_explicit(L, &D, S);
        if (schur_mode == 1) *pcg_iters = pcg_any(variant, L, &D, S, g, dc, pcg_max, pcg_tol, rel_res);
        else rc = dense_solve(S, m, g, dc);
        free(S);
    }
    if (!rc) back_substitute(L, &D, dc, dp);
    free(g); free(sb);
    damped_free(&D);
    return rc;
}

/* Public: one damped step from the given state (linearise + solve). */
int orc_step(int32_t nc, int32_t np, int64_t n, const double *cams, const double *pts, const double *obs,
             const int32_t *cam_idx, const int32_t *pt_idx, int loss, double delta, double mu, int damping,
             int schur_mode, int pcg_max, double pcg_tol, double *dc, double *dp, int *pcg_iters, double *rel_res,
             double *model_dec, int precond, const uint8_t *cam_fixed, const uint8_t *pt_fixed, int pcg_variant) {
    lin_t L;
    int rc = lin_alloc(&L, nc, np, n, cam_idx, pt_idx);
    if (rc) return rc;
    L.cam_fixed = cam_fixed;
    L.pt_fixed = pt_fixed;
    linearise(&L, cams, pts, obs, loss, delta);
    rc = damped_step(&L, mu, damping, schur_mode, pcg_max, pcg_tol, dc, dp, pcg_iters, rel_res, precond, NULL,
                     pcg_variant);
    if (!rc && model_dec) {
        double *scr = malloc(sizeof(double) * n);
        *model_dec = model_decrease(&L, dc, dp, scr);
        free(scr);
    }
    lin_free(&L);
    return rc;
}

/* Public: the Schur-Jacobi camera blocks S~_ii (nc*81, row-major) at damping mu. */
int orc_schur_jacobi_blocks(int32_t nc, int32_t np, int64_t n, const double *cams, const double *pts,
                            const double *obs, const int32_t *cam_idx, const int32_t *pt_idx, int loss, double delta,
                            double mu, int damping, double *blocks) {
    lin_t L;
    int rc = lin_alloc(&L, nc, np, n, cam_idx, pt_idx);
    if (rc) return rc;
    linearise(&L, cams, pts, obs, loss, delta);
    damped_t D;
    rc = damp(&L, mu, damping, &D);
    if (!rc) {
        schur_jacobi(&L, &D, blocks);
        damped_free(&D);
    }
    lin_free(&L);
    return rc;
}

/* Public: reduced-camera right-hand side and one implicit Schur product
 * y = S x at damping mu (Alg. 3), for checking a single matrix-vector step. */
int orc_schur(int32_t nc, int32_t np, int64_t n, const double *cams, const double *pts, const double *obs,
              const int32_t *cam_idx, const int32_t *pt_idx, int loss, double delta, double mu, int damping,
              const double *x, double *y, double *rhs, double *S_dense) {
    lin_t L;
    int rc = lin_alloc(&L, nc, np, n, cam_idx, pt_idx);
    if (rc) return rc;
    linearise(&L, cams, pts, obs, loss, delta);
    damped_t D;
    rc = damp(&L, mu, damping, &D);
    if (rc) { lin_free(&L); return rc; }
    double *sa = malloc(sizeof(double) * 3 * (size_t)np), *sb = malloc(sizeof(double) * 3 * (size_t)np);
    if (x && y) schur_matvec(&L, &D, x, y, sa, sb);
    if (rhs) schur_rhs(&L, &D, rhs, sb);
    if (S_dense) schur_explicit(&L, &D, S_dense);
    free(sa); free(sb);
    damped_free(&D);
    lin_free(&L);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the solved state (differentiable BA layer; the paper has no     */
/* counterpart).  At x* with M = H(x*) + mu D (the damped Gauss-Newton matrix */
/* of the last step), solve M v = gbar by the same Schur elimination and PCG  */
/* (gbar = dL/dx*, cameras then points).  By the implicit function theorem on */
/* the optimality condition J^T W e = 0 with e = pi(x) - u, d(x*) by du_k is  */
/* M^-1 J_k^T W_k, so dL/du_k = W_k J_k v (2 values per observation).  The    */
/* initial estimate enters through the damping of the last step (proximal     */
/* reading): dL/dx0 = mu D v.                                                 */
/* ------------------------------------------------------------------------ */
int orc_adjoint(int32_t nc, int32_t np, int64_t n, const double *cams, const double *pts, const double *obs,
                const int32_t *cam_idx, const int32_t *pt_idx, int loss, double delta, double mu, int damping,
                int pcg_max, double pcg_tol, const double *gbar_c, const double *gbar_p, double *grad_obs,
                double *grad_c0, double *grad_p0, int *pcg_iters, int precond, int pcg_variant) {
    lin_t L;
    int rc = lin_alloc(&L, nc, np, n, cam_idx, pt_idx);
    if (rc) return rc;
    linearise(&L, cams, pts, obs, loss, delta);
    /* diagonal damping terms D before the right-hand side is replaced */
    double *Dc = malloc(sizeof(double) * 9 * (size_t)nc), *Dp = malloc(sizeof(double) * 3 * (size_t)np);
    double *vc = malloc(sizeof(double) * 9 * (size_t)nc), *vp = malloc(sizeof(double) * 3 * (size_t)np);
    for (int32_t i = 0; i < nc; ++i)
        for (int a = 0; a < 9; ++a) Dc[9 * (int64_t)i + a] = damp_term(damping, L.Hpp[81 * (int64_t)i + a * 9 + a]);
    for (int32_t j = 0; j < np; ++j)
        for (int a = 0; a < 3; ++a) Dp[3 * (int64_t)j + a] = damp_term(damping, L.Hll[9 * (int64_t)j + a * 3 + a]);
    memcpy(L.v, gbar_c, sizeof(double) * 9 * (size_t)nc);
    memcpy(L.w, gbar_p, sizeof(double) * 3 * (size_t)np);
    int it = 0;
    rc = damped_step(&L, mu, damping, 0, pcg_max, pcg_tol, vc, vp, &it, NULL, precond, NULL, pcg_variant);
    if (!rc) {
        for (int64_t k = 0; k < n; ++k) {
            const double *Jc = L.Jc + 18 * k, *Jp = L.Jp + 6 * k;
            const double *xc = vc + 9 * (int64_t)cam_idx[k], *xp = vp + 3 * (int64_t)pt_idx[k];
            for (int r = 0; r < 2; ++r) {
                double s = 0.0;
                for (int a = 0; a < 9; ++a) s += Jc[r * 9 + a] * xc[a];
                for (int a = 0; a < 3; ++a) s += Jp[r * 3 + a] * xp[a];
                grad_obs[2 * k + r] = L.W[k] * s;
            }
        }
        for (int64_t t = 0; t < 9 * (int64_t)nc; ++t) grad_c0[t] = mu * Dc[t] * vc[t];
        for (int64_t t = 0; t < 3 * (int64_t)np; ++t) grad_p0[t] = mu * Dp[t] * vp[t];
        if (pcg_iters) *pcg_iters = it;
    }
    free(Dc); free(Dp); free(vc); free(vp);
    lin_free(&L);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Levenberg-Marquardt driver (Alg. 1 outer loop; Ceres-style trust region). */
/* Readings: radius starts at initial_radius, mu = 1/radius; step accepted    */
/* iff the model decrease is positive, the new cost is finite and the gain    */
/* ratio (F - F')/model_decrease exceeds min_rel_dec.  On acceptance          */
/* radius /= max(1/3, 1 - (2 rho - 1)^3) and the decrease factor resets to 2; */
/* on rejection radius /= factor and factor *= 2 (Nielsen's rule); radius is  */
/* clamped to [1e-32, 1e16].  A rejected iteration counts and reuses the     */
/* linearisation.  With function_tol > 0 the loop stops after an accepted     */
/* step whose |F - F'|/F < function_tol.  An iteration whose damped blocks */
/* are not all positive definite has no step and counts as rejected.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    double cost, cost_new, model_dec, mu, gain;
    int accepted, pcg_iters;
    double pcg_rel_res;
} orc_trace_t;

int orc_lm_solve(int32_t nc, int32_t np, int64_t n, double *cams, double *pts, const double *obs,
                 const int32_t *cam_idx, const int32_t *pt_idx, int loss, double delta, int max_iter, int pcg_max,
                 double pcg_tol, int damping, double initial_radius, double min_rel_dec, double function_tol,
                 int schur_mode, orc_trace_t *trace, int *iterations, double *final_cost, double *final_radius,
                 int precond, int forcing, const uint8_t *cam_fixed, const uint8_t *pt_fixed, int pcg_variant) {
    lin_t L;
    int rc = lin_alloc(&L, nc, np, n, cam_idx, pt_idx);
    if (rc) return rc;
    L.cam_fixed = cam_fixed;
    L.pt_fixed = pt_fixed;
    double *cand_c = malloc(sizeof(double) * 9 * (size_t)nc), *cand_p = malloc(sizeof(double) * 3 * (size_t)np);
    double *dc = malloc(sizeof(double) * 9 * (size_t)nc), *dp = malloc(sizeof(double) * 3 * (size_t)np);
    double *scr = malloc(sizeof(double) * (size_t)n);
    if (!cand_c || !cand_p || !dc || !dp || !scr) { rc = ORC_ERR_OOM; goto done; }

    double F = cost_only(n, cams, pts, obs, cam_idx, pt_idx, loss, delta, scr);
    double radius = initial_radius, factor = 2.0, g0n = 0.0;
    int relin = 1, it = 0;
    for (it = 0; it < max_iter; ++it) {
        if (relin) { linearise(&L, cams, pts, obs, loss, delta); relin = 0; }
        double mu = 1.0 / radius;
        int pcg_iters = 0;
        double rel_res = 0.0;
        rc = damped_step(&L, mu, damping, schur_mode, pcg_max, pcg_tol, dc, dp, &pcg_iters, &rel_res, precond,
                         forcing ? &g0n : NULL, pcg_variant);
        if (rc == ORC_ERR_NOT_SPD) {
            /* a damped block that is not positive definite gives no step: the
               iteration counts as rejected (mu grows, the linearisation is kept) */
            rc = ORC_OK;
            if (trace) {
                trace[it].cost = F; trace[it].cost_new = NAN; trace[it].model_dec = 0.0; trace[it].mu = mu;
                trace[it].gain = NAN; trace[it].accepted = 0; trace[it].pcg_iters = 0; trace[it].pcg_rel_res = 0.0;
            }
            radius = radius / factor;
            factor *= 2.0;
            if (radius < 1e-32) radius = 1e-32;
            continue;
        }
        if (rc) goto done;
        double ldec = model_decrease(&L, dc, dp, scr);
        for (int64_t t = 0; t < 9 * (int64_t)nc; ++t) cand_c[t] = cams[t] + dc[t];
        for (int64_t t = 0; t < 3 * (int64_t)np; ++t) cand_p[t] = pts[t] + dp[t];
        double Fn = cost_only(n, cand_c, cand_p, obs, cam_idx, pt_idx, loss, delta, scr);
        double gain = (F - Fn) / ldec;
        int accept = ldec > 0.0 && isfinite(Fn) && gain > min_rel_dec;
        if (trace) {
            trace[it].cost = F; trace[it].cost_new = Fn; trace[it].model_dec = ldec; trace[it].mu = mu;
            trace[it].gain = gain; trace[it].accepted = accept; trace[it].pcg_iters = pcg_iters;
            trace[it].pcg_rel_res = rel_res;
        }
        int stop = 0;
        if (accept) {
            double t = 2.0 * gain - 1.0;
            double shrink = 1.0 - t * t * t;
            radius = radius / (shrink > 1.0 / 3.0 ? shrink : 1.0 / 3.0);
            factor = 2.0;
            if (function_tol > 0.0 && fabs(F - Fn) < function_tol * F) stop = 1;
            memcpy(cams, cand_c, sizeof(double) * 9 * (size_t)nc);
            memcpy(pts, cand_p, sizeof(double) * 3 * (size_t)np);
            F = Fn;
            relin = 1;
        } else {
            radius = radius / factor;
            factor *= 2.0;
        }
        if (radius > 1e16) radius = 1e16;
        if (radius < 1e-32) radius = 1e-32;
        if (stop) { ++it; break; }
    }
    *iterations = it;
    *final_cost = F;
    *final_radius = radius;
done:
    free(cand_c); free(cand_p); free(dc); free(dp); free(scr);
    lin_free(&L);
    return rc;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
