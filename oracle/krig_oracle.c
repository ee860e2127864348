/*
 * krig_oracle.c -- plain, slow FP64 CPU oracle for ordinary kriging of the
 * missing inter-slice voxels of an MRI slice stack (arXiv 2303.09523).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path
 * is checked against.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline / reference leg may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * What it computes, and where the paper says so:
 *   - Sec. 4.1.1 and Algorithm 1 (steps 2-4): the stack of n known slices is
 *     cut along Z into k sub-blocks; each block is laid out as a partially
 *     filled 3-D matrix whose inter-slice gaps hold NaN ("Conc"); every NaN
 *     voxel is then filled by kriging; the blocks are merged back by their
 *     stored offsets (Sec. 4.2).
 *   - Sec. 4.1.2: the estimate is a weighted linear sum of known values whose
 *     weights minimise the estimation variance under an unbiasedness
 *     constraint, taken in 3-D over the neighbouring known voxels.
 *   - Appendix A (kriging with external drift, p predictors): with a single
 *     constant predictor q_1 = 1 the system is ordinary kriging: the weights
 *     and one Lagrange multiplier solve the extended (bordered) system.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - variogram models (absent from the paper): spherical, exponential with
 *     the practical range exp(-3h/a), and a linear model used only by pins;
 *     `sill` is the partial sill, gamma(0) = 0.
 *   - neighbourhood: the (2r+1)x(2r+1) in-plane window in each of the two
 *     bracketing known slices, truncated at the in-plane border.
 *   - coordinates: isotropic output grid; known slice j sits at z = j*g.
 *   - Z sub-blocks partition the gaps; neighbouring blocks share their
 *     boundary known slice.  The first (n-1) mod k blocks get one gap more.
 *   - the kriging variance is w^T gamma0 + mu (variogram form).
 *
 * The system is written in the variogram form
 *     [ Gamma 1 ] [ w  ]   [ gamma0 ]
 *     [ 1^T   0 ] [ mu ] = [ 1      ]
 * and solved by Gaussian elimination with partial pivoting, in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_get_max_threads(void) { return 1; }
#endif

typedef struct {
    int32_t model; /* 0 spherical, 1 exponential, 2 linear (pins only) */
    int32_t pad;
    double nugget;
    double sill;   /* partial sill */
    double range;  /* a */
} orc_variogram;

enum { ORC_SPHERICAL = 0, ORC_EXPONENTIAL = 1, ORC_LINEAR = 2 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ESINGULAR = 4 };

#define ORC_MAX_R 3
#define ORC_MAX_K (2 * (2 * ORC_MAX_R + 1) * (2 * ORC_MAX_R + 1))

/* ------------------------------------------------------------------------ */
/* Variogram and its partial derivatives w.r.t. (nugget, sill, range).       */
/* ------------------------------------------------------------------------ */

double orc_gamma(const orc_variogram* v, double h)
{
    if (h == 0.0) return 0.0; /* gamma(0) = 0 by definition of a semivariogram */
    double a = v->range;
    switch (v->model) {
    case ORC_SPHERICAL:
        if (h < a) {
            double q = h / a;
            return v->nugget + v->sill * (1.5 * q - 0.5 * q * q * q);
        }
        return v->nugget + v->sill;
    case ORC_EXPONENTIAL:
        return v->nugget + v->sill * (1.0 - exp(-3.0 * h / a));
    case ORC_LINEAR:
        return v->nugget + v->sill * h / a;
    }
    return NAN;
}

/* d gamma / d(nugget, sill, range) at lag h, written into d[3]. */
void orc_gamma_grad(const orc_variogram* v, double h, double d[3])
{
    d[0] = d[1] = d[2] = 0.0;
    if (h == 0.0) return;
    double a = v->range;
    d[0] = 1.0;
    switch (v->model) {
    case ORC_SPHERICAL:
        if (h < a) {
            double q = h / a;
            d[1] = 1.5 * q - 0.5 * q * q * q;
            /* d/da of 1.5 h/a - 0.5 h^3/a^3 = -1.5 h/a^2 + 1.5 h^3/a^4 */
            d[2] = v->sill * (-1.5 * h / (a * a) + 1.5 * h * h * h / (a * a * a * a));
        } else {
            d[1] = 1.0;
            d[2] = 0.0;
        }
        break;
    case ORC_EXPONENTIAL: {
        double e = exp(-3.0 * h / a);
        d[1] = 1.0 - e;
        /* d/da (1 - exp(-3h/a)) = -exp(-3h/a) * 3h / a^2 */
        d[2] = -v->sill * e * 3.0 * h / (a * a);
        break;
    }
    case ORC_LINEAR:
        d[1] = h / a;
        d[2] = -v->sill * h / (a * a);
        break;
    }
}

/* ------------------------------------------------------------------------ */
/* Dense Gaussian elimination with partial pivoting, m x m, nrhs columns.    */
/* A is row-major m x m, B is row-major m x nrhs; both are overwritten, the  */
/* solution is left in B.                                                    */
/* ------------------------------------------------------------------------ */

int orc_gauss_solve(int m, double* A, double* B, int nrhs)
{
    double amax = 0.0;
    for (int i = 0; i < m * m; ++i) amax = fmax(amax, fabs(A[i]));
    if (!(amax > 0.0)) return ORC_ESINGULAR;
    for (int k = 0; k < m; ++k) {
        int p = k;
        for (int i = k + 1; i < m; ++i)
            if (fabs(A[i * m + k]) > fabs(A[p * m + k])) p = i;
        if (!(fabs(A[p * m + k]) > 1e-13 * amax)) return ORC_ESINGULAR;
        if (p != k) {
            for (int j = 0; j < m; ++j) {
                double t = A[k * m + j]; A[k * m + j] = A[p * m + j]; A[p * m + j] = t;
            }
            for (int j = 0; j < nrhs; ++j) {
                double t = B[k * nrhs + j]; B[k * nrhs + j] = B[p * nrhs + j]; B[p * nrhs + j] = t;
            }
        }
        for (int i = k + 1; i < m; ++i) {
            double f = A[i * m + k] / A[k * m + k];
            if (f == 0.0) continue;
            for (int j = k; j < m; ++j) A[i * m + j] -= f * A[k * m + j];
            for (int j = 0; j < nrhs; ++j) B[i * nrhs + j] -= f * B[k * nrhs + j];
        }
    }
    for (int k = m - 1; k >= 0; --k) {
        for (int j = 0; j < nrhs; ++j) {
            double s = B[k * nrhs + j];
            for (int i = k + 1; i < m; ++i) s -= A[k * m + i] * B[i * nrhs + j];
            B[k * nrhs + j] = s / A[k * m + k];
        }
    }
    return ORC_OK;
}

static double dist3(const double* a, const double* b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* ------------------------------------------------------------------------ */
/* Ordinary kriging at one target s0 from K points (Appendix A, p = 1).      */
/*   pts: K x 3 coordinates; vals: K values (nullable).                      */
/*   Outputs (all nullable): w[K], mu, var, est.                             */
/*   dw: K x 3 derivative of the weights w.r.t. (nugget, sill, range),       */
/*   dvar: 3 derivatives of the variance (nullable).                          */
/* ------------------------------------------------------------------------ */

int orc_ok_solve(int K, const double* pts, const double* s0, const orc_variogram* v,
                 const double* vals, double* w, double* mu, double* var, double* est,
                 double* dw, double* dvar)
{
    if (K < 1 || K > ORC_MAX_K || !pts || !s0 || !v) return ORC_EINVAL;
    int m = K + 1;
    double* A = (double*)malloc(sizeof(double) * m * m * 2 + sizeof(double) * m * 4 + sizeof(double) * m);
    if (!A) return ORC_ENOMEM;
    double* A2 = A + m * m;
    double* B = A2 + m * m;     /* m x 4 */
    double* g0 = B + m * 4;     /* m */

    /* Gamma_ij = gamma(|s_i - s_j|), border of ones, corner 0. */
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j < K; ++j) A[i * m + j] = orc_gamma(v, dist3(pts + 3 * i, pts + 3 * j));
        A[i * m + K] = 1.0;
        A[K * m + i] = 1.0;
        g0[i] = orc_gamma(v, dist3(pts + 3 * i, s0));
    }
    A[K * m + K] = 0.0;
    g0[K] = 1.0;
    memcpy(A2, A, sizeof(double) * m * m);
    for (int i = 0; i < m; ++i) B[i] = g0[i];
    int st = orc_gauss_solve(m, A2, B, 1);
    if (st != ORC_OK) { free(A); return st; }
    /* B[0..K-1] = weights, B[K] = mu */
    double s_var = B[K], s_est = 0.0;
    for (int i = 0; i < K; ++i) {
        s_var += B[i] * g0[i];
        if (vals) s_est += B[i] * vals[i];
    }
    if (w) for (int i = 0; i < K; ++i) w[i] = B[i];
    if (mu) *mu = B[K];
    if (var) *var = s_var;
    if (est) *est = s_est;

    if (dw || dvar) {
        /* d lambda = A^{-1} (db - dA lambda) for each parameter p. */
        double* lam = (double*)malloc(sizeof(double) * m);
        double* R = (double*)malloc(sizeof(double) * m * 3);
        double* db = (double*)malloc(sizeof(double) * m * 3);
        if (!lam || !R || !db) { free(lam); free(R); free(db); free(A); return ORC_ENOMEM; }
        for (int i = 0; i < m; ++i) lam[i] = B[i];
        for (int i = 0; i < m * 3; ++i) db[i] = 0.0;
        for (int i = 0; i < K; ++i) orc_gamma_grad(v, dist3(pts + 3 * i, s0), db + 3 * i);
        for (int i = 0; i < m; ++i)
            for (int p = 0; p < 3; ++p) R[i * 3 + p] = db[i * 3 + p];
        for (int i = 0; i < K; ++i) {
            for (int j = 0; j < K; ++j) {
                double d[3];
                orc_gamma_grad(v, dist3(pts + 3 * i, pts + 3 * j), d);
                for (int p = 0; p < 3; ++p) R[i * 3 + p] -= d[p] * lam[j];
            }
        }
        memcpy(A2, A, sizeof(double) * m * m);
        st = orc_gauss_solve(m, A2, R, 3);
        if (st == ORC_OK) {
            if (dw)
                for (int i = 0; i < K; ++i)
                    for (int p = 0; p < 3; ++p) dw[i * 3 + p] = R[i * 3 + p];
            if (dvar) {
                /* var = sum_i w_i g0_i + mu */
                for (int p = 0; p < 3; ++p) {
                    double s = R[K * 3 + p];
                    for (int i = 0; i < K; ++i) s += R[i * 3 + p] * g0[i] + lam[i] * db[i * 3 + p];
                    dvar[p] = s;
                }
            }
        }
        free(lam); free(R); free(db);
    }
    free(A);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Neighbourhood of in-plane pixel (x, y) between two known slices          */
/* `lower` and `upper` (each H x W, row-major), which sit dz_lo below and    */
/* dz_hi above the target.  Window (2r+1)^2 in each slice, truncated at the  */
/* in-plane border.  Order: lower slice first, then rows dy, then dx.        */
/* ------------------------------------------------------------------------ */

static int gather(const double* lower, const double* upper, int H, int W, int x, int y,
                  int r, double dz_lo, double dz_hi, double* pts, double* vals)
{
    int K = 0;
    for (int s = 0; s < 2; ++s) {
        const double* sl = s == 0 ? lower : upper;
        double dz = s == 0 ? -dz_lo : dz_hi;
        for (int dy = -r; dy <= r; ++dy) {
            int yy = y + dy;
            if (yy < 0 || yy >= H) continue;
            for (int dx = -r; dx <= r; ++dx) {
                int xx = x + dx;
                if (xx < 0 || xx >= W) continue;
                pts[3 * K + 0] = (double)dx;
                pts[3 * K + 1] = (double)dy;
                pts[3 * K + 2] = dz;
                if (vals) vals[K] = sl[(size_t)yy * W + xx];
                ++K;
            }
        }
    }
    return K;
}

static const double s0_origin[3] = {0.0, 0.0, 0.0};

/* Estimate and variance at (x, y) between two known slices. */
static int predict(const double* lower, const double* upper, int H, int W, int x, int y, int r,
                   double dz_lo, double dz_hi, const orc_variogram* v, double* est, double* var)
{
    double pts[3 * ORC_MAX_K], vals[ORC_MAX_K];
    int K = gather(lower, upper, H, W, x, y, r, dz_lo, dz_hi, pts, vals);
    return orc_ok_solve(K, pts, s0_origin, v, vals, NULL, NULL, var, est, NULL, NULL);
}

/* Sub-block sizes: k blocks over G gaps, the first G mod k blocks one larger. */
static int64_t block_first_gap(int G, int k, int b)
{
    int q = G / k, rem = G % k;
    return (int64_t)b * q + (b < rem ? b : rem);
}

static int check_args(int n, int H, int W, int g, int r, const orc_variogram* v)
{
    if (n < 2 || H < 1 || W < 1 || g < 1 || r < 0 || r > ORC_MAX_R || !v) return 0;
    if (!(v->range > 0.0)) return 0;
    if (v->model < 0 || v->model > 2) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Whole volume (Algorithm 1, steps 2-4, and the merge of Sec. 4.2).         */
/*   slices: n x H x W.  out: ((n-1)g+1) x H x W.  var: same, nullable.      */
/*   k_sub: number of Z sub-blocks (1 <= k_sub <= n-1).                      */
/*   threads: OpenMP threads (0 = runtime default).                          */
/* ------------------------------------------------------------------------ */

int orc_krige_volume(const double* slices, int32_t n, int32_t H, int32_t W, int32_t g, int32_t r,
                     int32_t k_sub, const orc_variogram* v, int32_t threads, double* out,
                     double* var)
{
    if (!slices || !out || !check_args(n, H, W, g, r, v)) return ORC_EINVAL;
    int G = n - 1;
    if (k_sub < 1 || k_sub > G) return ORC_EINVAL;
    size_t plane = (size_t)H * W;
    int status = ORC_OK;

    for (int b = 0; b < k_sub; ++b) {
        int64_t a0 = block_first_gap(G, k_sub, b), a1 = block_first_gap(G, k_sub, b + 1);
        int gaps = (int)(a1 - a0);
        int depth = gaps * g + 1;
        /* Conc: a partially filled block, known slices every g, NaN between. */
        double* R = (double*)malloc(sizeof(double) * plane * depth);
        double* RV = (double*)malloc(sizeof(double) * plane * depth);
        if (!R || !RV) { free(R); free(RV); return ORC_ENOMEM; }
        for (size_t i = 0; i < plane * depth; ++i) { R[i] = NAN; RV[i] = 0.0; }
        for (int i = 0; i <= gaps; ++i)
            memcpy(R + (size_t)i * g * plane, slices + (size_t)(a0 + i) * plane, sizeof(double) * plane);

        /* Fill every NaN voxel of the block from its bracketing known slices. */
        int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : omp_get_max_threads()) reduction(| : bad)
        for (int64_t zy = 0; zy < (int64_t)depth * H; ++zy) {
            int z = (int)(zy / H), y = (int)(zy % H);
            for (int x = 0; x < W; ++x) {
                size_t idx = (size_t)z * plane + (size_t)y * W + x;
                if (!isnan(R[idx])) continue;
                int zl = (z / g) * g, zu = zl + g;
                double e, s2;
                int st = predict(R + (size_t)zl * plane, R + (size_t)zu * plane, H, W, x, y, r,
                                 (double)(z - zl), (double)(zu - z), v, &e, &s2);
                if (st != ORC_OK) { bad |= st; e = NAN; s2 = NAN; }
                R[idx] = e;
                RV[idx] = s2;
            }
        }
        if (bad) status = bad;
        /* Merge by stored offsets: block b starts at output slice a0*g. */
        memcpy(out + (size_t)a0 * g * plane, R, sizeof(double) * plane * depth);
        if (var) memcpy(var + (size_t)a0 * g * plane, RV, sizeof(double) * plane * depth);
        free(R);
        free(RV);
    }
    return status;
}

/* Selected output voxels only (for full-size parity on samples).            */
/*   zyx: count x 3 output coordinates (z in output slices).                  */
int orc_krige_voxels(const double* slices, int32_t n, int32_t H, int32_t W, int32_t g, int32_t r,
                     const orc_variogram* v, int64_t count, const int64_t* zyx, int32_t threads,
                     double* est, double* var)
{
    if (!slices || !zyx || !est || !check_args(n, H, W, g, r, v)) return ORC_EINVAL;
    int64_t nout = (int64_t)(n - 1) * g + 1;
    for (int64_t i = 0; i < count; ++i)
        if (zyx[3 * i] < 0 || zyx[3 * i] >= nout || zyx[3 * i + 1] < 0 || zyx[3 * i + 1] >= H ||
            zyx[3 * i + 2] < 0 || zyx[3 * i + 2] >= W)
            return ORC_EINVAL;
    size_t plane = (size_t)H * W;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads > 0 ? threads : omp_get_max_threads()) reduction(| : bad)
    for (int64_t i = 0; i < count; ++i) {
        int z = (int)zyx[3 * i], y = (int)zyx[3 * i + 1], x = (int)zyx[3 * i + 2];
        int j = z / g, t = z % g;
        double e, s2;
        if (t == 0) {
            e = slices[(size_t)j * plane + (size_t)y * W + x];
            s2 = 0.0;
        } else {
            int st = predict(slices + (size_t)j * plane, slices + (size_t)(j + 1) * plane, H, W, x, y,
                             r, (double)t, (double)(g - t), v, &e, &s2);
            if (st != ORC_OK) { bad |= st; e = NAN; s2 = NAN; }
        }
        est[i] = e;
        if (var) var[i] = s2;
    }
    return bad ? bad : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Leave-one-slice-out cross-validation (the differentiable fitting loss).   */
/* Interior known slice j (1..n-2) is predicted at its own z from slices     */
/* j-1 and j+1, which sit g below and g above it:                            */
/*     L = 1/((n-2) H W) * sum_j sum_{x,y} (zhat_j(x,y) - S_j(x,y))^2.        */
/* Outputs (nullable): loss, pred ((n-2) x H x W), grad_theta[3] =           */
/* dL/d(nugget, sill, range), grad_slices (n x H x W) = dL/dS.               */
/* ------------------------------------------------------------------------ */

int orc_loo(const double* slices, int32_t n, int32_t H, int32_t W, int32_t g, int32_t r,
            const orc_variogram* v, int32_t threads, double* loss, double* pred,
            double* grad_theta, double* grad_slices)
{
    if (!slices || !check_args(n, H, W, g, r, v) || n < 3) return ORC_EINVAL;
    size_t plane = (size_t)H * W;
    double N = (double)(n - 2) * (double)plane;
    double L = 0.0, gt0 = 0.0, gt1 = 0.0, gt2 = 0.0;
    int bad = 0;
    if (grad_slices) memset(grad_slices, 0, sizeof(double) * plane * n);
    int nthr = threads > 0 ? threads : omp_get_max_threads();
    /* Prediction j touches slices j-1, j, j+1 of grad_slices; predictions with
       j in the same residue class mod 3 touch disjoint slices. */
    for (int phase = 0; phase < 3; ++phase) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthr) reduction(+ : L, gt0, gt1, gt2) reduction(| : bad)
        for (int j = 1; j <= n - 2; ++j) {
            if (j % 3 != phase) continue;
            const double* lo = slices + (size_t)(j - 1) * plane;
            const double* hi = slices + (size_t)(j + 1) * plane;
            const double* tg = slices + (size_t)j * plane;
            double pts[3 * ORC_MAX_K], vals[ORC_MAX_K], w[ORC_MAX_K], dw[3 * ORC_MAX_K];
            for (int y = 0; y < H; ++y) {
                for (int x = 0; x < W; ++x) {
                    int K = gather(lo, hi, H, W, x, y, r, (double)g, (double)g, pts, vals);
                    double e;
                    int st = orc_ok_solve(K, pts, s0_origin, v, vals, w, NULL, NULL, &e,
                                          grad_theta ? dw : NULL, NULL);
                    if (st != ORC_OK) { bad |= st; continue; }
                    double res = e - tg[(size_t)y * W + x];
                    L += res * res;
                    if (pred) pred[(size_t)(j - 1) * plane + (size_t)y * W + x] = e;
                    if (grad_theta) {
                        double d0 = 0, d1 = 0, d2 = 0;
                        for (int k = 0; k < K; ++k) {
                            d0 += dw[3 * k + 0] * vals[k];
                            d1 += dw[3 * k + 1] * vals[k];
                            d2 += dw[3 * k + 2] * vals[k];
                        }
                        gt0 += 2.0 * res * d0 / N;
                        gt1 += 2.0 * res * d1 / N;
                        gt2 += 2.0 * res * d2 / N;
                    }
                    if (grad_slices) {
                        /* zhat = sum_k w_k S(neighbour k): scatter 2 res w_k / N;
                           the target enters with -1. */
                        int k = 0;
                        for (int s = 0; s < 2; ++s) {
                            double* gs = grad_slices + (size_t)(s == 0 ? j - 1 : j + 1) * plane;
                            for (int dy = -r; dy <= r; ++dy) {
                                int yy = y + dy;
                                if (yy < 0 || yy >= H) continue;
                                for (int dx = -r; dx <= r; ++dx) {
                                    int xx = x + dx;
                                    if (xx < 0 || xx >= W) continue;
                                    gs[(size_t)yy * W + xx] += 2.0 * res * w[k] / N;
                                    ++k;
                                }
                            }
                        }
                        grad_slices[(size_t)j * plane + (size_t)y * W + x] -= 2.0 * res / N;
                    }
                }
            }
        }
    }
    if (loss) *loss = L / N;
    if (grad_theta) { grad_theta[0] = gt0; grad_theta[1] = gt1; grad_theta[2] = gt2; }
    return bad ? bad : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Universal kriging / kriging with external drift (Appendix A, p > 1).      */
/*                                                                          */
/* The weights honour sum_i w_i q_k(s_i) = q_k(s0) for every predictor q_k    */
/* (Appendix A's constraint), one Lagrange multiplier each, in the variogram */
/* form                                                                     */
/*     [ Gamma  F ] [ w  ]   [ gamma0 ]                                      */
/*     [ F^T    0 ] [ mu ] = [ f0     ],  F_ik = q_k(s_i), f0_k = q_k(s0),    */
/* and the kriging variance is w^T gamma0 + mu^T f0.  Predictors here are    */
/* polynomial drifts in the coordinates (the paper names universal kriging   */
/* without saying which): drift 0 = {1} (ordinary kriging), 1 = {1, z},      */
/* 2 = {1, x, y, z}.                                                         */
/* ------------------------------------------------------------------------ */

#define ORC_MAX_SLABS 4
#define ORC_UK_MAX_K (ORC_MAX_SLABS * (2 * ORC_MAX_R + 1) * (2 * ORC_MAX_R + 1))

static int drift_terms(int drift) { return drift == 0 ? 1 : (drift == 1 ? 2 : 4); }

static void drift_row(int drift, const double* s, double* q)
{
    q[0] = 1.0;
    if (drift == 1) {
        q[1] = s[2];
    } else if (drift == 2) {
        q[1] = s[0];
        q[2] = s[1];
        q[3] = s[2];
    }
}

int orc_uk_solve(int K, const double* pts, const double* s0, const orc_variogram* v, int drift,
                 const double* vals, double* w, double* mu, double* var, double* est)
{
    if (K < 1 || K > ORC_UK_MAX_K || !pts || !s0 || !v || drift < 0 || drift > 2) return ORC_EINVAL;
    const int p = drift_terms(drift), m = K + p;
    double* A = (double*)malloc(sizeof(double) * ((size_t)m * m + 2 * (size_t)m));
    if (!A) return ORC_ENOMEM;
    double* B = A + (size_t)m * m;
    double* g0 = B + m;
    double q[4], q0[4];
    drift_row(drift, s0, q0);
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j < K; ++j) A[i * m + j] = orc_gamma(v, dist3(pts + 3 * i, pts + 3 * j));
        drift_row(drift, pts + 3 * i, q);
        for (int k = 0; k < p; ++k) {
            A[i * m + K + k] = q[k];
            A[(K + k) * m + i] = q[k];
        }
        g0[i] = orc_gamma(v, dist3(pts + 3 * i, s0));
    }
    for (int k = 0; k < p; ++k) {
        for (int l = 0; l < p; ++l) A[(K + k) * m + K + l] = 0.0;
        g0[K + k] = q0[k];
    }
    for (int i = 0; i < m; ++i) B[i] = g0[i];
    int st = orc_gauss_solve(m, A, B, 1);
    if (st != ORC_OK) { free(A); return st; }
    double s_var = 0.0, s_est = 0.0;
    for (int i = 0; i < m; ++i) s_var += B[i] * g0[i];  /* w^T gamma0 + mu^T f0 */
    if (vals)
        for (int i = 0; i < K; ++i) s_est += B[i] * vals[i];
    if (w) for (int i = 0; i < K; ++i) w[i] = B[i];
    if (mu) for (int k = 0; k < p; ++k) mu[k] = B[K + k];
    if (var) *var = s_var;
    if (est) *est = s_est;
    free(A);
    return ORC_OK;
}

/* Neighbourhood over `slabs` known slices (2: j, j+1; 4: j-1 .. j+2, those
 * that exist) of a target in gap j at offset t, window (2r+1)^2 truncated at
 * the in-plane border; coordinates relative to the target. */
static int gather_slabs(const double* slices, int n, int H, int W, int g, int j, int t, int x, int y, int r,
                        int slabs, double* pts, double* vals)
{
    const size_t plane = (size_t)H * W;
    const int first = slabs == 4 ? j - 1 : j, last = slabs == 4 ? j + 2 : j + 1;
    int K = 0;
    for (int jj = first; jj <= last; ++jj) {
        if (jj < 0 || jj >= n) continue;
        const double dz = (double)(jj - j) * g - t;
        for (int dy = -r; dy <= r; ++dy) {
            const int yy = y + dy;
            if (yy < 0 || yy >= H) continue;
            for (int dx = -r; dx <= r; ++dx) {
                const int xx = x + dx;
                if (xx < 0 || xx >= W) continue;
                pts[3 * K + 0] = (double)dx;
                pts[3 * K + 1] = (double)dy;
                pts[3 * K + 2] = dz;
                vals[K] = slices[(size_t)jj * plane + (size_t)yy * W + xx];
                ++K;
            }
        }
    }
    return K;
}

/* Universal kriging at sampled output voxels (z, y, x) of the (n-1)g+1 slice
 * output: known slices copied, missing voxels predicted from `slabs` known
 * slices with the given drift.  est, var: count values (var nullable). */
int orc_uk_voxels(const double* slices, int32_t n, int32_t H, int32_t W, int32_t g, int32_t r, int32_t slabs,
                  int32_t drift, const orc_variogram* v, int64_t count, const int64_t* zyx, double* est, double* var)
{
    if (!slices || !zyx || !est || !check_args(n, H, W, g, r, v) || (slabs != 2 && slabs != 4) || drift < 0 ||
        drift > 2)
        return ORC_EINVAL;
    const int64_t nout = (int64_t)(n - 1) * g + 1;
    for (int64_t i = 0; i < count; ++i)
        if (zyx[3 * i] < 0 || zyx[3 * i] >= nout || zyx[3 * i + 1] < 0 || zyx[3 * i + 1] >= H ||
            zyx[3 * i + 2] < 0 || zyx[3 * i + 2] >= W)
            return ORC_EINVAL;
    const size_t plane = (size_t)H * W;
    int bad = 0;
    for (int64_t i = 0; i < count; ++i) {
        const int z = (int)zyx[3 * i], y = (int)zyx[3 * i + 1], x = (int)zyx[3 * i + 2];
        const int j = z / g, t = z % g;
        double e, s2;
        if (t == 0) {
            e = slices[(size_t)j * plane + (size_t)y * W + x];
            s2 = 0.0;
        } else {
            double pts[3 * ORC_UK_MAX_K], vals[ORC_UK_MAX_K];
            const int K = gather_slabs(slices, n, H, W, g, j, t, x, y, r, slabs, pts, vals);
            const int st = orc_uk_solve(K, pts, s0_origin, v, drift, vals, NULL, NULL, &s2, &e);
            if (st != ORC_OK) { bad |= st; e = NAN; s2 = NAN; }
        }
        est[i] = e;
        if (var) var[i] = s2;
    }
    return bad ? bad : ORC_OK;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
