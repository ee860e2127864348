// krig_uk.cu -- universal kriging (Appendix A with more than one predictor) of
// the missing voxels: the class solve and the stencil apply.
//
// Appendix A writes the weights of kriging with external drift as the solution
// of the extended system with one unbiasedness constraint and one Lagrange
// multiplier per predictor q_k; Sec. 4.1.2 calls the method universal kriging
// and speaks of "all possible 64 neighbours" of a voxel.  The predictors are not
// named; this path takes polynomial drift in the voxel coordinates, {1, z} or
// {1, x, y, z} ({1} is ordinary kriging), and a neighbourhood of two known
// slices (the bracketing pair) or four (one more on each side, where it exists).
//
// Geometry classes: the system of a missing voxel depends only on its offset t
// in the gap, on how its (2r+1)^2 window is truncated at the in-plane border,
// and, with four slabs, on which of the outer slices exist (the first gap has
// none below, the last none above).  In coordinates relative to the gap's lower
// known slice the point-to-point covariances and the drift rows do not depend
// on t either, so each class is one Cholesky factorisation shared by all g-1
// targets (FP32 factor, two refinement steps with float-float residuals) (the drift basis {1, x, y, z - t} of the target-centred system
// and {1, x, y, z} span the same functions, so the weights are the same).
//
// Covariance form (C(h) = nugget + sill - gamma(h), SPD for a valid model):
//   C w + F lambda = c0,  F' w = f0   =>   w = C^-1 (c0 - F lambda),
//   S lambda = F' C^-1 c0 - f0 with S = F' C^-1 F,
//   kriging variance C(0) - w'c0 - f0'lambda  (= w'gamma0 + mu'f0 of the
//   variogram form).
// The stencil kernel applies each class's weights from shared-memory tiles of
// the slabs of one gap, and copies the known slices through.
#include <cuda_runtime.h>
#include <stdint.h>

#include "krig_device.cuh"

#define UK_MAXS 4
#define UK_KMAX (UK_MAXS * (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1))  // 100 points
#define UK_PMAX 4
#define UK_NRHS (KRIG_GMAX - 1 + UK_PMAX)                           // c0 of every t, then F
#define UK_THREADS 256

namespace {

// Slab s of a gap: known slice j + s - 1 with four slabs, j + s with two; its z
// relative to slice j.
__host__ __device__ inline int uk_slab_dj(int slabs, int s) { return slabs == 4 ? s - 1 : s; }

// Dynamic shared memory of the class solve.
struct UkSolveSmem {
    ff A[UK_KMAX * UK_KMAX];      // C as float-float pairs (for the refinement residuals)
    double X[UK_KMAX * UK_NRHS];  // right-hand sides [i][col], then the solutions
    double c0[UK_KMAX * (KRIG_GMAX - 1)];
    double pt[UK_KMAX][3];
    double S[UK_PMAX * UK_PMAX];
    double lam[KRIG_GMAX - 1][UK_PMAX];
    double var[KRIG_GMAX - 1];
    // covariance at every distinct lag between two points: [slab distance][|dy|][|dx|]
    ff lag[UK_MAXS][2 * KRIG_RMAX + 1][2 * KRIG_RMAX + 1];
    ff B[UK_KMAX * UK_NRHS];       // the right-hand sides [c0 | F], kept for the residuals
    ff Xf[UK_KMAX * UK_NRHS];      // the solution during the refinement
    float L[UK_KMAX * UK_KMAX];    // FP32 Cholesky factor of C (lower)
    float Z[UK_KMAX * UK_NRHS];    // FP32 sweep operand
    float col[UK_KMAX];            // the current column of the factorisation
    int tap[UK_KMAX];             // (s * n2r + dy + r) * n2r + dx + r in the full window
    int ok;
};

__device__ void uk_sync() { __syncthreads(); }

}  // namespace

__global__ void __launch_bounds__(UK_THREADS) k_uk_solve(const __grid_constant__ KrigLaunch P)
{
    extern __shared__ __align__(16) unsigned char uk_smem[];
    UkSolveSmem& M = *(UkSolveSmem*)uk_smem;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the volume of this class block
    const int64_t cls = blockIdx.x;
    int v = 0;
    for (int u = 1; u < P.n_vols; ++u)
        if (P.vol[u].uk_cls_begin <= cls && P.vol[u].g >= 2) v = u;
    const KrigVol& V = P.vol[v];
    if (V.g < 2) return;
    const int slabs = P.uk_slabs, drift = P.uk_drift, p = krig_uk_terms(drift);
    const int local = (int)(cls - V.uk_cls_begin);
    const int cx = local % V.ncx, cy = (local / V.ncx) % V.ncy, pat = local / (V.ncx * V.ncy);
    const int r = V.r, n2r = 2 * r + 1, g = V.g, G1 = g - 1;
    const int lx = V.xext[cx][0], rx = V.xext[cx][1], ly = V.yext[cy][0], ry = V.yext[cy][1];
    const krig_variogram vg = P.vg[v];
    // points in order (slab, dy, dx), present slabs only
    if (tid == 0) {
        int K = 0;
        for (int s = 0; s < slabs; ++s) {
            if (slabs == 4 && ((s == 0 && (pat & 1)) || (s == 3 && (pat & 2)))) continue;
            for (int dy = -ly; dy <= ry; ++dy)
                for (int dx = -lx; dx <= rx; ++dx) {
                    M.pt[K][0] = dx;
                    M.pt[K][1] = dy;
                    M.pt[K][2] = (double)uk_slab_dj(slabs, s) * g;
                    M.tap[K] = (s * n2r + dy + r) * n2r + dx + r;
                    ++K;
                }
        }
        M.ok = K;
    }
    uk_sync();
    const int K = M.ok;
    const int NR = G1 + p;
    // C from one covariance evaluation per distinct lag (slab distance, |dy|, |dx|):
    // the same squared lag, hence the same value, as an evaluation per entry
    for (int e = tid; e < UK_MAXS * n2r * n2r; e += UK_THREADS) {
        const int ax = e % n2r, ay = (e / n2r) % n2r, ds = e / (n2r * n2r);
        const double dx = ax, dy = ay, dz = (double)ds * g;
        M.lag[ds][ay][ax] = ff_from_double(krig_cov(vg, dx * dx + dy * dy + dz * dz));
    }
    uk_sync();
    for (int e = tid; e < K * K; e += UK_THREADS) {
        const int i = e / K, j = e % K;
        const int ax = abs((int)M.pt[i][0] - (int)M.pt[j][0]), ay = abs((int)M.pt[i][1] - (int)M.pt[j][1]);
        const int ds = abs(M.tap[i] / (n2r * n2r) - M.tap[j] / (n2r * n2r));  // slab distance
        M.A[i * K + j] = M.lag[ds][ay][ax];
    }
    // the right-hand sides c0(t) and the drift columns F
    for (int e = tid; e < K * G1; e += UK_THREADS) {
        const int i = e / G1, t = e % G1 + 1;
        const double dz = M.pt[i][2] - t;
        const double c = krig_cov(vg, M.pt[i][0] * M.pt[i][0] + M.pt[i][1] * M.pt[i][1] + dz * dz);
        M.c0[i * G1 + t - 1] = c;
        M.X[i * UK_NRHS + t - 1] = c;
    }
    for (int e = tid; e < K * p; e += UK_THREADS) {
        const int i = e / p, k = e % p;
        double f = 1.0;
        if (drift == 1 && k == 1) f = M.pt[i][2];
        if (drift == 2 && k > 0) f = M.pt[i][k - 1];
        M.X[i * UK_NRHS + G1 + k] = f;
    }
    uk_sync();
    // C X = [c0 | F] by an FP32 Cholesky factorisation and two refinement steps with
    // float-float residuals (FP64 issues at 1/64 of the FP32 rate on this GPU; C
    // and the right-hand sides are kept as pairs for the residuals)
    for (int e = tid; e < K * K; e += UK_THREADS) M.L[e] = M.A[e].hi;
    for (int e = tid; e < K * NR; e += UK_THREADS) {
        const int i = e / NR, c = e % NR;
        M.B[i * UK_NRHS + c] = ff_from_double(M.X[i * UK_NRHS + c]);
    }
    uk_sync();
    bool ok = true;
    for (int k = 0; k < K; ++k) {
        const float d = M.L[k * K + k];
        if (!(d > 0.0f)) {  // the same value in every thread
            ok = false;
            break;
        }
        const float l = sqrtf(d), il = 1.0f / l;
        uk_sync();
        for (int i = k + 1 + tid; i < K; i += UK_THREADS) {
            const float v = M.L[i * K + k] * il;
            M.L[i * K + k] = v;
            M.col[i] = v;
        }
        if (tid == 0) M.L[k * K + k] = l;
        uk_sync();
        // trailing update of the lower triangle: rows i, columns j <= i (16 x 16 thread grid)
        for (int i = k + 1 + (tid >> 4); i < K; i += 16) {
            const float li = M.col[i];
            for (int j = k + 1 + (tid & 15); j <= i; j += 16) M.L[i * K + j] = fmaf(-li, M.col[j], M.L[i * K + j]);
        }
        uk_sync();
    }
    // Z <- C^-1 Z by the FP32 factor, every column at once (thread grid: 16 rows x 16 columns)
    auto sweeps = [&]() {
        for (int i = 0; i < K; ++i) {
            if (tid < NR) M.Z[i * UK_NRHS + tid] /= M.L[i * K + i];
            uk_sync();
            if ((tid & 15) < NR)
                for (int k2 = i + 1 + (tid >> 4); k2 < K; k2 += 16)
                    M.Z[k2 * UK_NRHS + (tid & 15)] =
                        fmaf(-M.L[k2 * K + i], M.Z[i * UK_NRHS + (tid & 15)], M.Z[k2 * UK_NRHS + (tid & 15)]);
            uk_sync();
        }
        for (int i = K - 1; i >= 0; --i) {
            if (tid < NR) M.Z[i * UK_NRHS + tid] /= M.L[i * K + i];
            uk_sync();
            if ((tid & 15) < NR)
                for (int k2 = (tid >> 4); k2 < i; k2 += 16)
                    M.Z[k2 * UK_NRHS + (tid & 15)] =
                        fmaf(-M.L[i * K + k2], M.Z[i * UK_NRHS + (tid & 15)], M.Z[k2 * UK_NRHS + (tid & 15)]);
            uk_sync();
        }
    };
    if (!ok) {
        if (tid == 0) krig_set_status(P.status, KRIG_DEV_SINGULAR);
    } else {
        for (int e = tid; e < K * NR; e += UK_THREADS) {
            const int i = e / NR, c = e % NR;
            M.Z[i * UK_NRHS + c] = M.B[i * UK_NRHS + c].hi;
        }
        uk_sync();
        sweeps();
        for (int e = tid; e < K * NR; e += UK_THREADS) {
            const int i = e / NR, c = e % NR;
            M.Xf[i * UK_NRHS + c] = ff_make(M.Z[i * UK_NRHS + c]);
        }
        uk_sync();
        for (int it = 0; it < 2; ++it) {
            // R = [c0 | F] - C X compensated (Dot2 over the pairs; the low part of X
            // enters the compensation), then X += C^-1 R in FP32
            for (int e = tid; e < K * NR; e += UK_THREADS) {
                const int i = e / NR, c = e % NR;
                ff_dot acc(M.B[i * UK_NRHS + c]);
                for (int j = 0; j < K; ++j) {
                    const ff a = M.A[i * K + j], x = M.Xf[j * UK_NRHS + c];
                    acc.add(a, -x.hi);
                    acc.c = __fmaf_rn(-a.hi, x.lo, acc.c);
                }
                M.Z[i * UK_NRHS + c] = ff_round(acc.value());
            }
            uk_sync();
            sweeps();
            for (int e = tid; e < K * NR; e += UK_THREADS) {
                const int i = e / NR, c = e % NR;
                M.Xf[i * UK_NRHS + c] = ff_add(M.Xf[i * UK_NRHS + c], ff_make(M.Z[i * UK_NRHS + c]));
            }
            uk_sync();
        }
        for (int e = tid; e < K * NR; e += UK_THREADS) {
            const int i = e / NR, c = e % NR;
            M.X[i * UK_NRHS + c] = ff_to_double(M.Xf[i * UK_NRHS + c]);
        }
        uk_sync();
        // S = F' C^-1 F, and per target the multipliers: S lambda = F' C^-1 c0 - f0
        if (tid < p * p) {
            const int a = tid / p, b = tid % p;
            double s = 0.0;
            for (int i = 0; i < K; ++i) {
                double fa = 1.0;
                if (drift == 1 && a == 1) fa = M.pt[i][2];
                if (drift == 2 && a > 0) fa = M.pt[i][a - 1];
                s += fa * M.X[i * UK_NRHS + G1 + b];
            }
            M.S[a * p + b] = s;
        }
        uk_sync();
        if (tid < G1) {
            const int t = tid + 1;
            double rhs[UK_PMAX], S[UK_PMAX][UK_PMAX];
            for (int a = 0; a < p; ++a) {
                double s = 0.0;
                for (int i = 0; i < K; ++i) s += M.X[i * UK_NRHS + G1 + a] * M.c0[i * G1 + t - 1];  // F'C^-1 c0
                double f0 = a == 0 ? 1.0 : 0.0;
                if ((drift == 1 && a == 1) || (drift == 2 && a == 3)) f0 = (double)t;
                rhs[a] = s - f0;
                for (int b = 0; b < p; ++b) S[a][b] = M.S[a * p + b];
            }
            // Gaussian elimination with partial pivoting on the p x p system
            bool good = true;
            for (int k = 0; k < p; ++k) {
                int piv = k;
                for (int i = k + 1; i < p; ++i)
                    if (fabs(S[i][k]) > fabs(S[piv][k])) piv = i;
                if (!(fabs(S[piv][k]) > 0.0)) {
                    good = false;
                    break;
                }
                for (int b = 0; b < p; ++b) {
                    const double tmp = S[k][b];
                    S[k][b] = S[piv][b];
                    S[piv][b] = tmp;
                }
                const double tr = rhs[k];
                rhs[k] = rhs[piv];
                rhs[piv] = tr;
                for (int i = k + 1; i < p; ++i) {
                    const double f = S[i][k] / S[k][k];
                    for (int b = k; b < p; ++b) S[i][b] -= f * S[k][b];
                    rhs[i] -= f * rhs[k];
                }
            }
            for (int k = p - 1; k >= 0 && good; --k) {
                double s = rhs[k];
                for (int b = k + 1; b < p; ++b) s -= S[k][b] * M.lam[t - 1][b];
                M.lam[t - 1][k] = s / S[k][k];
            }
            if (!good) {
                krig_set_status(P.status, KRIG_DEV_SINGULAR);
                for (int k = 0; k < p; ++k) M.lam[t - 1][k] = __longlong_as_double(0x7ff8000000000000LL);
            }
        }
        uk_sync();
        // weights w_t = C^-1 c0_t - (C^-1 F) lambda_t, kept in the c0 columns of X
        for (int e = tid; e < K * G1; e += UK_THREADS) {
            const int i = e / G1, t = e % G1 + 1;
            double w = M.X[i * UK_NRHS + t - 1];
            for (int k = 0; k < p; ++k) w -= M.X[i * UK_NRHS + G1 + k] * M.lam[t - 1][k];
            M.X[i * UK_NRHS + t - 1] = w;
        }
        uk_sync();
        if (tid < G1) {
            const int t = tid + 1;
            double s = 0.0;
            for (int i = 0; i < K; ++i) s += M.X[i * UK_NRHS + t - 1] * M.c0[i * G1 + t - 1];
            double fl = M.lam[t - 1][0];
            if (drift == 1) fl += t * M.lam[t - 1][1];
            if (drift == 2) fl += t * M.lam[t - 1][3];
            M.var[t - 1] = (vg.nugget + vg.sill) - s - fl;
        }
    }
    uk_sync();
    // the class's row of the weight and variance tables (zeros on absent taps and
    // slabs; uint16 input: the weights carry the scale)
    const int ntap = slabs * n2r * n2r;
    const double scale = V.dtype == KRIG_U16 ? (double)V.scale : 1.0;
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    const int64_t row = (int64_t)local * ntap * KRIG_TSLOTS;
    for (int e = tid; e < ntap * KRIG_TSLOTS; e += UK_THREADS) {
        const int c = e % KRIG_TSLOTS, f = e / KRIG_TSLOTS;
        double w = 0.0;
        if (c < G1) {
            for (int i = 0; i < K; ++i)
                if (M.tap[i] == f) w = ok ? M.X[i * UK_NRHS + c] * scale : qnan;
        }
        if (V.dtype == KRIG_F64) ((double*)(P.ws + V.uk_wtab_off))[row + e] = w;
        else ((float*)(P.ws + V.uk_wtab_off))[row + e] = (float)w;
    }
    if (tid < KRIG_TSLOTS) {
        float* vt = (float*)(P.ws + V.uk_vtab_off) + (int64_t)local * KRIG_TSLOTS;
        vt[tid] = tid < G1 ? (ok ? (float)M.var[tid] : __int_as_float(0x7fc00000)) : 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Stencil apply: one block per (volume, gap, 32 x 16 tile).  The gap's slabs
// (tile plus halo, zeros outside the stack) are staged in shared memory; each
// thread computes two pixels of one row, every target t of the gap: interior
// pixels through per-slab D4 orbit sums and the interior class's orbit weights
// (staged in shared memory), border pixels through the full weight row of their
// class (read through L1).  The block also copies the gap's lower known slice
// (and the stack's last one) to the output.
// ---------------------------------------------------------------------------
template <typename TI> struct UkT { typedef float TC; typedef float TO; };
template <> struct UkT<double> { typedef double TC; typedef double TO; };

__device__ __forceinline__ float uk_cvt(float x, float) { return x; }
__device__ __forceinline__ double uk_cvt(double x, float) { return x; }
__device__ __forceinline__ float uk_cvt(uint16_t u, float) { return (float)u; }

// D4 orbit of tap (dx, dy): {same max(|dx|,|dy|), min(|dx|,|dy|)}, numbered a (a + 1) / 2 + b.
__host__ __device__ constexpr int uk_orbit(int dx, int dy)
{
    const int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy;
    const int a = ax > ay ? ax : ay, b = ax > ay ? ay : ax;
    return a * (a + 1) / 2 + b;
}

// One block per (volume, gap j, 32 x 16 tile): the gap's slabs staged in shared
// memory, each thread two pixels, every target t of the gap.  The interior class
// is invariant under the in-plane symmetries of the square (its window is full
// and the drift space {1, x, y, z} is mapped onto itself by them), so its
// weights are constant on each D4 orbit of every slab: interior pixels take
// orbit sums per slab and one weight per (slab, orbit, t), the orbit's member
// (dx, dy) = (a, b) of the solved row; the other classes take their full rows.
template <typename TI, int R, int GM1>
__device__ __forceinline__ void uk_apply_block(const KrigLaunch& P, int v, int j, int tile, unsigned char* smem)
{
    typedef typename UkT<TI>::TC TC;
    typedef typename UkT<TI>::TO TO;
    constexpr int N2R = 2 * R + 1, TW = KRIG_UK_TX + 2 * R, TH = KRIG_UK_TY + 2 * R;
    constexpr int NO = (R + 1) * (R + 2) / 2;
    const KrigVol& V = P.vol[v];
    const int slabs = P.uk_slabs, H = V.H, W = V.W, g = V.g, n = V.n;
    const int x0 = (tile % V.uk_tiles_x) * KRIG_UK_TX, y0 = (tile / V.uk_tiles_x) * KRIG_UK_TY;
    const int64_t plane = (int64_t)H * W;
    const TI* in = (const TI*)P.in[v];
    TC* tiles = (TC*)smem;                                  // [slabs][TH][TW]
    TC* wint = tiles + UK_MAXS * TH * TW;                   // interior weights per orbit [slabs][NO][8]
    const int pat = slabs == 4 ? ((j == 0 ? 1 : 0) | (j + 2 > n - 1 ? 2 : 0)) : 0;
    const int ntap = slabs * N2R * N2R;
    for (int e = threadIdx.x; e < slabs * TH * TW; e += UK_THREADS) {
        const int s = e / (TH * TW), rr = (e / TW) % TH, cc = e % TW;
        const int jj = j + uk_slab_dj(slabs, s), yy = y0 - R + rr, xx = x0 - R + cc;
        TC val = TC(0);
        if (jj >= 0 && jj < n && yy >= 0 && yy < H && xx >= 0 && xx < W)
            val = (TC)uk_cvt(in[(size_t)jj * plane + (size_t)yy * W + xx], V.scale);
        tiles[e] = val;
    }
    const int64_t cls_base = (int64_t)pat * V.ncy * V.ncx;
    const TC* wtab = (const TC*)(P.ws + V.uk_wtab_off);
    const float* vtab = (const float*)(P.ws + V.uk_vtab_off);
    if (V.cint >= 0)
        for (int e = threadIdx.x; e < slabs * NO * KRIG_TSLOTS; e += UK_THREADS) {
            const int t = e % KRIG_TSLOTS, o = (e / KRIG_TSLOTS) % NO, s = e / (KRIG_TSLOTS * NO);
            int a = 0;
            while ((a + 1) * (a + 2) / 2 <= o) ++a;
            const int b = o - a * (a + 1) / 2;  // member (dx, dy) = (a, b)
            wint[e] = wtab[(cls_base + V.cint) * ntap * KRIG_TSLOTS + ((s * N2R + (b + R)) * N2R + (a + R)) * KRIG_TSLOTS + t];
        }
    __syncthreads();
    const int row = threadIdx.x >> 4, col = (threadIdx.x & 15) * 2;
    const int y = y0 + row;
    if (y >= H) return;
    TO* out = (TO*)P.out[v];
    float* var = P.var[v];
    const int sj = slabs == 4 ? 1 : 0;  // slab of known slice j
    for (int q = 0; q < 2; ++q) {
        const int x = x0 + col + q;
        if (x >= W) continue;
        const int64_t pix = (int64_t)y * W + x;
        // known slice j (and the last one after the last gap), bit-exact
        const TC kv = tiles[(sj * TH + row + R) * TW + col + q + R];
        out[(int64_t)j * g * plane + pix] = (TO)(sizeof(TI) == 2 ? __fmul_rn((float)kv, V.scale) : kv);
        if (var) var[(int64_t)j * g * plane + pix] = 0.0f;
        if (j == n - 2) {
            const TC kl = tiles[((sj + 1) * TH + row + R) * TW + col + q + R];
            out[(int64_t)(j + 1) * g * plane + pix] = (TO)(sizeof(TI) == 2 ? __fmul_rn((float)kl, V.scale) : kl);
            if (var) var[(int64_t)(j + 1) * g * plane + pix] = 0.0f;
        }
        if constexpr (GM1 > 0) {
            const int cy = V.ymap[krig_slot(y, H, R)], cx = V.xmap[krig_slot(x, W, R)];
            const int64_t cls = cls_base + (int64_t)cy * V.ncx + cx;
            TC acc[GM1];
#pragma unroll
            for (int t = 0; t < GM1; ++t) acc[t] = TC(0);
            if (cy * V.ncx + cx == V.cint) {
#pragma unroll
                for (int s = 0; s < UK_MAXS; ++s) {
                    if (s >= slabs) break;
                    TC orb[NO];
#pragma unroll
                    for (int o = 0; o < NO; ++o) orb[o] = TC(0);
#pragma unroll
                    for (int dy = 0; dy < N2R; ++dy)
#pragma unroll
                        for (int dx = 0; dx < N2R; ++dx)
                            orb[uk_orbit(dx - R, dy - R)] += tiles[(s * TH + row + dy) * TW + col + q + dx];
#pragma unroll
                    for (int o = 0; o < NO; ++o) {
                        const TC* wr = wint + (s * NO + o) * KRIG_TSLOTS;
#pragma unroll
                        for (int t = 0; t < GM1; ++t) acc[t] = fma(wr[t], orb[o], acc[t]);
                    }
                }
            } else {
                const TC* w = wtab + cls * ntap * KRIG_TSLOTS;
                for (int s = 0; s < slabs; ++s)
#pragma unroll
                    for (int dy = 0; dy < N2R; ++dy)
#pragma unroll
                        for (int dx = 0; dx < N2R; ++dx) {
                            const TC z = tiles[(s * TH + row + dy) * TW + col + q + dx];
                            const TC* wr = w + ((s * N2R + dy) * N2R + dx) * KRIG_TSLOTS;
#pragma unroll
                            for (int t = 0; t < GM1; ++t) acc[t] = fma(wr[t], z, acc[t]);
                        }
            }
            const float* vr = vtab + cls * KRIG_TSLOTS;
#pragma unroll
            for (int t = 0; t < GM1; ++t) {
                out[((int64_t)j * g + t + 1) * plane + pix] = (TO)acc[t];
                if (var) var[((int64_t)j * g + t + 1) * plane + pix] = vr[t];
            }
        }
    }
}

template <typename TI, int R>
__device__ __forceinline__ void uk_apply_g(const KrigLaunch& P, int v, int g, int j, int tile, unsigned char* smem)
{
    switch (g) {
    case 1: uk_apply_block<TI, R, 0>(P, v, j, tile, smem); break;
    case 2: uk_apply_block<TI, R, 1>(P, v, j, tile, smem); break;
    case 3: uk_apply_block<TI, R, 2>(P, v, j, tile, smem); break;
    case 4: uk_apply_block<TI, R, 3>(P, v, j, tile, smem); break;
    case 5: uk_apply_block<TI, R, 4>(P, v, j, tile, smem); break;
    case 6: uk_apply_block<TI, R, 5>(P, v, j, tile, smem); break;
    case 7: uk_apply_block<TI, R, 6>(P, v, j, tile, smem); break;
    default: uk_apply_block<TI, R, 7>(P, v, j, tile, smem); break;
    }
}

template <typename TI>
__global__ void __launch_bounds__(UK_THREADS) k_uk_apply(const __grid_constant__ KrigLaunch P)
{
    extern __shared__ __align__(16) unsigned char uk_smem[];
    const int dtype = sizeof(TI) == 8 ? KRIG_F64 : sizeof(TI) == 4 ? KRIG_F32 : KRIG_U16;
    const int64_t it = blockIdx.x;
    int v = 0;
    for (int u = 1; u < P.n_vols; ++u)
        if (P.vol[u].uk_item_begin <= it) v = u;
    const KrigVol& V = P.vol[v];
    if (V.dtype != dtype) return;
    const int tiles = V.uk_tiles_x * V.uk_tiles_y;
    const int local = (int)(it - V.uk_item_begin);
    const int j = local / tiles, tile = local % tiles;
    switch (V.r) {
    case 0: uk_apply_g<TI, 0>(P, v, V.g, j, tile, uk_smem); break;
    case 1: uk_apply_g<TI, 1>(P, v, V.g, j, tile, uk_smem); break;
    default: uk_apply_g<TI, 2>(P, v, V.g, j, tile, uk_smem); break;
    }
}

template <typename TI>
static size_t uk_apply_smem()
{
    typedef typename UkT<TI>::TC TC;
    constexpr int TW = KRIG_UK_TX + 2 * KRIG_RMAX, TH = KRIG_UK_TY + 2 * KRIG_RMAX;
    return (size_t)(UK_MAXS * TH * TW + UK_KMAX * KRIG_TSLOTS) * sizeof(TC);
}

template <typename TI>
static int uk_launch_apply(const KrigLaunch& L, cudaStream_t st)
{
    const int dtype = sizeof(TI) == 8 ? KRIG_F64 : sizeof(TI) == 4 ? KRIG_F32 : KRIG_U16;
    bool any = false;
    for (int v = 0; v < L.n_vols; ++v) any = any || L.vol[v].dtype == dtype;
    if (!any || L.n_uk_items == 0) return 0;
    const size_t smem = uk_apply_smem<TI>();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_uk_apply<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    k_uk_apply<TI><<<(unsigned)L.n_uk_items, UK_THREADS, smem, st>>>(L);
    return (int)cudaGetLastError();
}

int krig_launch_uk(const KrigLaunch& L, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (L.n_uk_classes > 0) {
        const size_t smem = sizeof(UkSolveSmem);
        cudaError_t e = cudaFuncSetAttribute(k_uk_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        k_uk_solve<<<(unsigned)L.n_uk_classes, UK_THREADS, smem, st>>>(L);
        e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    int e = uk_launch_apply<float>(L, st);
    if (!e) e = uk_launch_apply<uint16_t>(L, st);
    if (!e) e = uk_launch_apply<double>(L, st);
    return e;
}
