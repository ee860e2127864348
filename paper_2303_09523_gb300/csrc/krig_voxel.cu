// krig_voxel.cu -- the per-voxel forms of the kriging path.
//
// Every missing voxel gathers its own neighbourhood (the (2r+1)^2 window in
// each bracketing known slice, truncated at the in-plane border), builds its
// own extended ordinary-kriging system (Appendix A with one constant
// predictor), solves it and forms the weighted sum and the kriging variance
// (Sec. 4.1.2).  One warp per voxel.
//   P64: FP64 Cholesky factorisation and solves.
//   PMX: FP32 factorisation and solves plus one FP64 iterative-refinement step.
// The covariances at the few distinct lags of a volume are tabulated once per
// call in FP64 (k_lag) and looked up while each voxel builds its matrix.
#include <cuda_runtime.h>
#include <stdint.h>

#include "krig_device.cuh"

__global__ void __launch_bounds__(256) k_lag(const __grid_constant__ KrigLaunch P)
{
    const int v = blockIdx.x;
    const KrigVol& V = P.vol[v];
    if (V.g < 2) return;
    LagDims d{V.r, V.g, 2 * V.r + 1, V.r + 1};
    double* gC = (double*)(P.ws + V.lag_off);
    double* g0 = gC + d.nC();
    const krig_variogram vg = P.vg[v];
    krig_fill_lags(d, vg, gC, g0, threadIdx.x, 256);
}

__device__ __forceinline__ double in_value(const void* in, int dtype, float scale, int64_t idx)
{
    if (dtype == KRIG_F64) return ((const double*)in)[idx];
    if (dtype == KRIG_F32) return (double)((const float*)in)[idx];
    return (double)__fmul_rn((float)((const uint16_t*)in)[idx], scale);
}

// Register factorisation for PMX at every size and for P64 up to 18 points;
// the FP64 50-point factor (200 registers) stays in shared memory.
template <typename TF, int KM>
struct VoxKind {
    static constexpr bool REG = sizeof(TF) == 4 || KM <= 18;
};

template <typename TF, int KM, bool REG>
struct VoxSmemSel;
template <typename TF, int KM>
struct VoxSmemSel<TF, KM, true> { typedef VoxSmem<KM, TF> type; };
template <typename TF, int KM>
struct VoxSmemSel<TF, KM, false> { typedef SolveSmem<TF, KM, 2> type; };

template <typename TF, int KM>
using VoxSmemT = typename VoxSmemSel<TF, KM, VoxKind<TF, KM>::REG>::type;

template <typename TF, int RMAX>
struct VoxSmemMax {
    static constexpr size_t s2 = sizeof(VoxSmemT<TF, 2>);
    static constexpr size_t s18 = RMAX >= 1 ? sizeof(VoxSmemT<TF, 18>) : 0;
    static constexpr size_t s50 = RMAX >= 2 ? sizeof(VoxSmemT<TF, 50>) : 0;
    static constexpr size_t m1 = s2 > s18 ? s2 : s18;
    static constexpr size_t bytes = ((m1 > s50 ? m1 : s50) + 15) / 16 * 16;
};

// Solve one voxel's system with the solver for its window size KM; S.Xd gets
// u and v.  The solver depends only on the voxel's own half-width, so a voxel
// gives the same bits whatever other volumes share the launch.
template <typename TF, int KM>
__device__ __forceinline__ bool voxel_solve(unsigned char* raw, const LagDims& d, const double* gC, const double* g0,
                                            int t, int lx, int rx, int ly, int ry, int lane, Tap** tap_out,
                                            double** bd_out, double** xd_out)
{
    typedef VoxSmemT<TF, KM> Smem;
    Smem& S = *(Smem*)raw;
    const int nx = lx + rx + 1, ny = ly + ry + 1;
    const int K = 2 * nx * ny;
    __syncwarp();
    for (int i = lane; i < K; i += 32) {
        Tap tp;
        tp.s = (int8_t)(i / (nx * ny));
        tp.dy = (int8_t)((i / nx) % ny - ly);
        tp.dx = (int8_t)(i % nx - lx);
        tp.pad = 0;
        S.tap[i] = tp;
        S.Bd[i * 2 + 0] = __ldg(g0 + d.i0(t, tp.s, abs((int)tp.dy), abs((int)tp.dx)));
        S.Bd[i * 2 + 1] = 1.0;
    }
    __syncwarp();
    *tap_out = S.tap;
    *bd_out = S.Bd;
    *xd_out = S.Xd;
    if constexpr (VoxKind<TF, KM>::REG) return warp_ok_solve_vox<KM, TF>(S, d, gC, K, lane);
    else return team_ok_solve<TF, KM, 2, 32>(S, d, gC, K, 2, lane);
}

template <typename TF, int RMAX>
__global__ void __launch_bounds__(256) k_voxel(const __grid_constant__ KrigLaunch P, int rmin)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* raw = smraw + (size_t)warp * VoxSmemMax<TF, RMAX>::bytes;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t vox = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; vox < P.n_vox; vox += nwarps) {
        const int v = krig_find_vol(P, vox, 2);
        const KrigVol& V = P.vol[v];
        const int64_t local = vox - V.vox_begin;
        const int64_t plane = (int64_t)V.H * V.W;
        const int z = (int)(local / plane);
        const int64_t pix = local % plane;
        const int y = (int)(pix / V.W), x = (int)(pix % V.W);
        const int g = V.g, j = z / g, t = z % g;
        const bool f64 = V.dtype == KRIG_F64;
        if (V.r < rmin) continue;  // voxel of the one-voxel-per-lane kernel
        if (t == 0) {  // known slice: copy through
            if (lane == 0) {
                double val = in_value(P.in[v], V.dtype, V.scale, (int64_t)j * plane + pix);
                if (f64) ((double*)P.out[v])[local] = val;
                else ((float*)P.out[v])[local] = (float)val;
                if (P.var[v]) P.var[v][local] = 0.0f;
            }
            continue;
        }
        const int r = V.r;
        LagDims d{r, g, 2 * r + 1, r + 1};
        const double* gC = (const double*)(P.ws + V.lag_off);
        const double* g0 = gC + d.nC();
        const int lx = min(x, r), rx = min(V.W - 1 - x, r), ly = min(y, r), ry = min(V.H - 1 - y, r);
        const int K = 2 * (lx + rx + 1) * (ly + ry + 1);
        Tap* tap;
        double *Bd, *Xd;
        bool ok;
        if (RMAX == 0 || r == 0) ok = voxel_solve<TF, 2>(raw, d, gC, g0, t, lx, rx, ly, ry, lane, &tap, &Bd, &Xd);
        else if (RMAX == 1 || r == 1) ok = voxel_solve<TF, 18>(raw, d, gC, g0, t, lx, rx, ly, ry, lane, &tap, &Bd, &Xd);
        else ok = voxel_solve<TF, (RMAX >= 2 ? 50 : 18)>(raw, d, gC, g0, t, lx, rx, ly, ry, lane, &tap, &Bd, &Xd);
        double est = 0.0, var = 0.0;
        if (ok) {
            double su = 0.0, sv = 0.0;
            for (int i = lane; i < K; i += 32) {
                su += Xd[i * 2 + 0];
                sv += Xd[i * 2 + 1];
            }
            for (int o = 16; o; o >>= 1) {
                su += __shfl_xor_sync(0xffffffffu, su, o);
                sv += __shfl_xor_sync(0xffffffffu, sv, o);
            }
            const double phi = (su - 1.0) / sv;
            double wz = 0.0, wc = 0.0;
            for (int i = lane; i < K; i += 32) {
                Tap tp = tap[i];
                double w = Xd[i * 2 + 0] - phi * Xd[i * 2 + 1];
                int64_t idx = (int64_t)(j + tp.s) * plane + (int64_t)(y + tp.dy) * V.W + (x + tp.dx);
                wz += w * in_value(P.in[v], V.dtype, V.scale, idx);
                wc += w * Bd[i * 2 + 0];
            }
            for (int o = 16; o; o >>= 1) {
                wz += __shfl_xor_sync(0xffffffffu, wz, o);
                wc += __shfl_xor_sync(0xffffffffu, wc, o);
            }
            est = wz;
            var = gC[0] - wc - phi;
        } else {
            est = var = __longlong_as_double(0x7ff8000000000000LL);
            if (lane == 0) krig_set_status(P.status, KRIG_DEV_SINGULAR);
        }
        if (lane == 0) {
            if (f64) ((double*)P.out[v])[local] = est;
            else ((float*)P.out[v])[local] = (float)est;
            if (P.var[v]) P.var[v][local] = (float)var;
        }
    }
}


// ---------------------------------------------------------------------------
// P64 for windows of up to 18 points (r <= 1): one voxel per lane.  A warp
// of FP64 work per voxel leaves most lanes idle on an 18-point system; here
// every lane factors its own voxel's system, so each FP64 instruction does
// 32 voxels' work.  LDL' factorisation (C is SPD, no pivoting) of the lower
// triangle in shared memory, interleaved [element][lane] so that the lanes
// of a warp touch consecutive words; u = C^-1 c0 and v = C^-1 1 by forward,
// diagonal and backward sweeps, then phi, w, the estimate and the variance as
// in the warp kernel.  The voxel's result does not depend on which other
// volumes share the launch.
// ---------------------------------------------------------------------------
constexpr int LK = 18, LT = LK * (LK + 1) / 2;  // points, lower-triangle entries
constexpr int LWARPS = 4;                       // warps per block
constexpr size_t LSMEM = (size_t)LWARPS * (LT + 2 * LK) * 32 * sizeof(double);

__global__ void __launch_bounds__(LWARPS * 32, 1) k_voxel_lane(const __grid_constant__ KrigLaunch P)
{
    extern __shared__ __align__(16) double lsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* const Lm = lsm + (size_t)warp * (LT + 2 * LK) * 32;
    double* const bu = Lm + LT * 32;
    double* const bv = bu + LK * 32;
#define LE(e) Lm[(e) * 32 + lane]
#define BU(i) bu[(i) * 32 + lane]
#define BV(i) bv[(i) * 32 + lane]
    const int64_t stride = (int64_t)gridDim.x * LWARPS * 32;
    for (int64_t vox = ((int64_t)blockIdx.x * LWARPS + warp) * 32 + lane; vox < P.n_vox; vox += stride) {
        const int v = krig_find_vol(P, vox, 2);
        const KrigVol& V = P.vol[v];
        const int r = V.r;
        if (r > 1) continue;  // voxel of the warp-per-voxel kernel
        const int64_t local = vox - V.vox_begin;
        const int64_t plane = (int64_t)V.H * V.W;
        const int z = (int)(local / plane);
        const int64_t pix = local % plane;
        const int y = (int)(pix / V.W), x = (int)(pix % V.W);
        const int g = V.g, j = z / g, t = z % g;
        const bool f64 = V.dtype == KRIG_F64;
        if (t == 0) {  // known slice: copy through
            const double val = in_value(P.in[v], V.dtype, V.scale, (int64_t)j * plane + pix);
            if (f64) ((double*)P.out[v])[local] = val;
            else ((float*)P.out[v])[local] = (float)val;
            if (P.var[v]) P.var[v][local] = 0.0f;
            continue;
        }
        LagDims d{r, g, 2 * r + 1, r + 1};
        const double* gC = (const double*)(P.ws + V.lag_off);
        const double* g0 = gC + d.nC();
        const int lx = min(x, r), rx = min(V.W - 1 - x, r), ly = min(y, r), ry = min(V.H - 1 - y, r);
        const int nx = lx + rx + 1, ny = ly + ry + 1, nxy = nx * ny;
        const int K = 2 * nxy;
        // system (lower triangle, row-major) and right-hand sides; point i is
        // (slice i / nxy, dy = (i / nx) % ny - ly, dx = i % nx - lx)
        for (int i = 0; i < K; ++i) {
            const int si = i / nxy, dyi = (i / nx) % ny - ly, dxi = i % nx - lx;
            for (int k = 0; k <= i; ++k) {
                const int sk = k / nxy, dyk = (k / nx) % ny - ly, dxk = k % nx - lx;
                LE(i * (i + 1) / 2 + k) = __ldg(gC + d.iC(si != sk, abs(dyi - dyk), abs(dxi - dxk)));
            }
            BU(i) = __ldg(g0 + d.i0(t, si, abs(dyi), abs(dxi)));
            BV(i) = 1.0;
        }
        // LDL': column k of L below the diagonal replaces a_ik, 1/d_k replaces a_kk
        bool ok = true;
        for (int k = 0; k < K && ok; ++k) {
            const int kk = k * (k + 1) / 2;
            const double dk = LE(kk + k);
            if (!(dk > 0.0)) {
                ok = false;
                break;
            }
            const double inv = 1.0 / dk;
            LE(kk + k) = inv;
            for (int i = k + 1; i < K; ++i) {
                const int ii = i * (i + 1) / 2;
                const double ti = LE(ii + k);  // unscaled a_ik
                const double li = ti * inv;
                LE(ii + k) = li;
#pragma unroll 4
                for (int jj = k + 1; jj < i; ++jj) LE(ii + jj) = fma(-ti, LE(jj * (jj + 1) / 2 + k), LE(ii + jj));
                LE(ii + i) = fma(-ti, li, LE(ii + i));
            }
        }
        double est, var;
        if (ok) {
            // L y = b (unit lower), then D z = y, then L' x = z, for u and v at once
            for (int i = 1; i < K; ++i) {
                const int ii = i * (i + 1) / 2;
                double au = BU(i), av = BV(i);
#pragma unroll 4
                for (int k = 0; k < i; ++k) {
                    const double l = LE(ii + k);
                    au = fma(-l, BU(k), au);
                    av = fma(-l, BV(k), av);
                }
                BU(i) = au;
                BV(i) = av;
            }
            for (int i = 0; i < K; ++i) {
                const double inv = LE(i * (i + 1) / 2 + i);
                BU(i) *= inv;
                BV(i) *= inv;
            }
            for (int i = K - 2; i >= 0; --i) {
                double au = BU(i), av = BV(i);
#pragma unroll 4
                for (int k = i + 1; k < K; ++k) {
                    const double l = LE(k * (k + 1) / 2 + i);
                    au = fma(-l, BU(k), au);
                    av = fma(-l, BV(k), av);
                }
                BU(i) = au;
                BV(i) = av;
            }
            double su = 0.0, sv = 0.0;
            for (int i = 0; i < K; ++i) {
                su += BU(i);
                sv += BV(i);
            }
            const double phi = (su - 1.0) / sv;
            double wz = 0.0, wc = 0.0;
            for (int i = 0; i < K; ++i) {
                const int si = i / nxy, dyi = (i / nx) % ny - ly, dxi = i % nx - lx;
                const double w = BU(i) - phi * BV(i);
                const int64_t idx = (int64_t)(j + si) * plane + (int64_t)(y + dyi) * V.W + (x + dxi);
                wz += w * in_value(P.in[v], V.dtype, V.scale, idx);
                wc += w * __ldg(g0 + d.i0(t, si, abs(dyi), abs(dxi)));
            }
            est = wz;
            var = gC[0] - wc - phi;
        } else {
            est = var = __longlong_as_double(0x7ff8000000000000LL);
            krig_set_status(P.status, KRIG_DEV_SINGULAR);
        }
        if (f64) ((double*)P.out[v])[local] = est;
        else ((float*)P.out[v])[local] = (float)est;
        if (P.var[v]) P.var[v][local] = (float)var;
    }
#undef LE
#undef BU
#undef BV
}

// ---------------------------------------------------------------------------
// PMX for windows of up to 18 points: one voxel per lane, as k_voxel_lane, but
// the factorisation and the sweeps in FP32 and one step of FP64 iterative
// refinement: x0 = C^-1 b in FP32, the residual b - C x0 in FP64 (C and b
// from the FP64 lag tables), the correction by the FP32 factors, x = x0 + d
// in FP64; then phi, w, the estimate and the variance in FP64.  The FP64 work
// per voxel is the residual (2 K^2 FMAs) and the combine, against the K^3/6 +
// 2 K^2 of the plain FP64 form.
// ---------------------------------------------------------------------------
constexpr int MWARPS = 6;
constexpr size_t MSMEM = (size_t)MWARPS * 32 * (LT * sizeof(float) + 2 * LK * sizeof(double) + 2 * LK * sizeof(float));

__global__ void __launch_bounds__(MWARPS * 32, 1) k_voxel_lane_mx(const __grid_constant__ KrigLaunch P)
{
    extern __shared__ __align__(16) unsigned char msm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = msm + (size_t)warp * 32 * (LT * sizeof(float) + 2 * LK * sizeof(double) + 2 * LK * sizeof(float));
    float* const Lm = (float*)base;                       // [LT][32] factor
    double* const xu = (double*)(Lm + LT * 32);           // [LK][32] solutions (FP64)
    double* const xv = xu + LK * 32;
    float* const ru = (float*)(xv + LK * 32);             // [LK][32] sweep vectors (FP32)
    float* const rv = ru + LK * 32;
#define LE(e) Lm[(e) * 32 + lane]
#define XU(i) xu[(i) * 32 + lane]
#define XV(i) xv[(i) * 32 + lane]
#define RU(i) ru[(i) * 32 + lane]
#define RV(i) rv[(i) * 32 + lane]
    const int64_t stride = (int64_t)gridDim.x * MWARPS * 32;
    for (int64_t vox = ((int64_t)blockIdx.x * MWARPS + warp) * 32 + lane; vox < P.n_vox; vox += stride) {
        const int v = krig_find_vol(P, vox, 2);
        const KrigVol& V = P.vol[v];
        const int r = V.r;
        if (r > 1) continue;  // voxel of the warp-per-voxel kernel
        const int64_t local = vox - V.vox_begin;
        const int64_t plane = (int64_t)V.H * V.W;
        const int z = (int)(local / plane);
        const int64_t pix = local % plane;
        const int y = (int)(pix / V.W), x = (int)(pix % V.W);
        const int g = V.g, j = z / g, t = z % g;
        const bool f64 = V.dtype == KRIG_F64;
        if (t == 0) {  // known slice: copy through
            const double val = in_value(P.in[v], V.dtype, V.scale, (int64_t)j * plane + pix);
            if (f64) ((double*)P.out[v])[local] = val;
            else ((float*)P.out[v])[local] = (float)val;
            if (P.var[v]) P.var[v][local] = 0.0f;
            continue;
        }
        LagDims d{r, g, 2 * r + 1, r + 1};
        const double* gC = (const double*)(P.ws + V.lag_off);
        const double* g0 = gC + d.nC();
        const int lx = min(x, r), rx = min(V.W - 1 - x, r), ly = min(y, r), ry = min(V.H - 1 - y, r);
        const int nx = lx + rx + 1, ny = ly + ry + 1, nxy = nx * ny;
        const int K = 2 * nxy;
        // FP32 system (lower triangle) and right-hand sides
        for (int i = 0; i < K; ++i) {
            const int si = i / nxy, dyi = (i / nx) % ny - ly, dxi = i % nx - lx;
            for (int k = 0; k <= i; ++k) {
                const int sk = k / nxy, dyk = (k / nx) % ny - ly, dxk = k % nx - lx;
                LE(i * (i + 1) / 2 + k) = (float)__ldg(gC + d.iC(si != sk, abs(dyi - dyk), abs(dxi - dxk)));
            }
            RU(i) = (float)__ldg(g0 + d.i0(t, si, abs(dyi), abs(dxi)));
            RV(i) = 1.0f;
        }
        // FP32 LDL'
        bool ok = true;
        for (int k = 0; k < K && ok; ++k) {
            const int kk = k * (k + 1) / 2;
            const float dk = LE(kk + k);
            if (!(dk > 0.0f)) {
                ok = false;
                break;
            }
            const float inv = 1.0f / dk;
            LE(kk + k) = inv;
            for (int i = k + 1; i < K; ++i) {
                const int ii = i * (i + 1) / 2;
                const float ti = LE(ii + k);
                const float li = ti * inv;
                LE(ii + k) = li;
#pragma unroll 4
                for (int jj = k + 1; jj < i; ++jj) LE(ii + jj) = fmaf(-ti, LE(jj * (jj + 1) / 2 + k), LE(ii + jj));
                LE(ii + i) = fmaf(-ti, li, LE(ii + i));
            }
        }
        double est, var;
        if (ok) {
            // x = C^-1 b with the FP32 factors, applied to (RU, RV) in place
            auto sweep = [&]() {
                for (int i = 1; i < K; ++i) {
                    const int ii = i * (i + 1) / 2;
                    float au = RU(i), av = RV(i);
#pragma unroll 4
                    for (int k = 0; k < i; ++k) {
                        const float l = LE(ii + k);
                        au = fmaf(-l, RU(k), au);
                        av = fmaf(-l, RV(k), av);
                    }
                    RU(i) = au;
                    RV(i) = av;
                }
                for (int i = 0; i < K; ++i) {
                    const float inv = LE(i * (i + 1) / 2 + i);
                    RU(i) *= inv;
                    RV(i) *= inv;
                }
                for (int i = K - 2; i >= 0; --i) {
                    float au = RU(i), av = RV(i);
#pragma unroll 4
                    for (int k = i + 1; k < K; ++k) {
                        const float l = LE(k * (k + 1) / 2 + i);
                        au = fmaf(-l, RU(k), au);
                        av = fmaf(-l, RV(k), av);
                    }
                    RU(i) = au;
                    RV(i) = av;
                }
            };
            sweep();
            for (int i = 0; i < K; ++i) {
                XU(i) = (double)RU(i);
                XV(i) = (double)RV(i);
            }
            // one FP64 refinement step: residual b - C x in FP64, corrected by the FP32 factors
            for (int i = 0; i < K; ++i) {
                const int si = i / nxy, dyi = (i / nx) % ny - ly, dxi = i % nx - lx;
                double au = __ldg(g0 + d.i0(t, si, abs(dyi), abs(dxi))), av = 1.0;
                for (int k = 0; k < K; ++k) {
                    const int sk = k / nxy, dyk = (k / nx) % ny - ly, dxk = k % nx - lx;
                    const double c = __ldg(gC + d.iC(si != sk, abs(dyi - dyk), abs(dxi - dxk)));
                    au = fma(-c, XU(k), au);
                    av = fma(-c, XV(k), av);
                }
                RU(i) = (float)au;
                RV(i) = (float)av;
            }
            sweep();
            double su = 0.0, sv = 0.0;
            for (int i = 0; i < K; ++i) {
                XU(i) += (double)RU(i);
                XV(i) += (double)RV(i);
                su += XU(i);
                sv += XV(i);
            }
            const double phi = (su - 1.0) / sv;
            double wz = 0.0, wc = 0.0;
            for (int i = 0; i < K; ++i) {
                const int si = i / nxy, dyi = (i / nx) % ny - ly, dxi = i % nx - lx;
                const double w = XU(i) - phi * XV(i);
                const int64_t idx = (int64_t)(j + si) * plane + (int64_t)(y + dyi) * V.W + (x + dxi);
                wz += w * in_value(P.in[v], V.dtype, V.scale, idx);
                wc += w * __ldg(g0 + d.i0(t, si, abs(dyi), abs(dxi)));
            }
            est = wz;
            var = gC[0] - wc - phi;
        } else {
            est = var = __longlong_as_double(0x7ff8000000000000LL);
            krig_set_status(P.status, KRIG_DEV_SINGULAR);
        }
        if (f64) ((double*)P.out[v])[local] = est;
        else ((float*)P.out[v])[local] = (float)est;
        if (P.var[v]) P.var[v][local] = (float)var;
    }
#undef LE
#undef XU
#undef XV
#undef RU
#undef RV
}

template <typename TF, int RMAX>
static int launch_voxel_t(const KrigLaunch& L, cudaStream_t st, int rmin)
{
    const size_t smem = 8 * VoxSmemMax<TF, RMAX>::bytes;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_voxel<TF, RMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_voxel<TF, RMAX>, 256, smem);
    if (e != cudaSuccess) return (int)e;
    int sms = krig_device_sm_count();
    int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    int64_t need = (L.n_vox + 7) / 8;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_voxel<TF, RMAX><<<(unsigned)grid, 256, smem, st>>>(L, rmin);
    return (int)cudaGetLastError();
}

static int launch_voxel_lane(const KrigLaunch& L, cudaStream_t st, bool mixed)
{
    const int warps = mixed ? MWARPS : LWARPS;
    const size_t smem = mixed ? MSMEM : LSMEM;
    cudaError_t e = mixed ? cudaFuncSetAttribute(k_voxel_lane_mx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                          : cudaFuncSetAttribute(k_voxel_lane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    const int sms = krig_device_sm_count();
    int64_t grid = sms > 0 ? sms : 1;
    const int64_t need = (L.n_vox + warps * 32 - 1) / (warps * 32);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    if (mixed) k_voxel_lane_mx<<<(unsigned)grid, warps * 32, smem, st>>>(L);
    else k_voxel_lane<<<(unsigned)grid, warps * 32, smem, st>>>(L);
    return (int)cudaGetLastError();
}

int krig_launch_voxel(const KrigLaunch& L, int form, void* stream)
{
    if (L.n_vox == 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    k_lag<<<L.n_vols, 256, 0, st>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    int rmax = 0;
    for (int v = 0; v < L.n_vols; ++v) rmax = L.vol[v].r > rmax ? L.vol[v].r : rmax;
    const bool fp64 = form == KRIG_FORM_P64;
    // voxels of volumes with r <= 1: one per lane; r = 2: one per warp
    int rmin = 0;
    for (int v = 0; v < L.n_vols; ++v) rmin = (v == 0 || L.vol[v].r < rmin) ? L.vol[v].r : rmin;
    if (rmin <= 1) {
        const int rc = launch_voxel_lane(L, st, !fp64);
        if (rc) return rc;
    }
    if (rmax < 2) return 0;
    return fp64 ? launch_voxel_t<double, 2>(L, st, 2) : launch_voxel_t<float, 2>(L, st, 2);
}
