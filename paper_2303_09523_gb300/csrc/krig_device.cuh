// krig_device.cuh -- device building blocks shared by the kriging kernels:
// the covariance model, the lag tables and the ordinary-kriging solver.
//
// The solver works in the covariance form of the extended system of
// Appendix A with one constant predictor (ordinary kriging):
//     [ C  1 ] [ w   ]   [ c0 ]
//     [ 1' 0 ] [ phi ] = [ 1  ],   C_ij = C(|s_i - s_j|), c0_i = C(|s_i - s0|),
// with C(h) = nugget + sill - gamma(h).  C is symmetric positive definite for
// a valid model and distinct points, so the bordered system is solved by a
// Cholesky factorisation of C and the Schur complement of the border:
//     u = C^-1 c0,  v = C^-1 1,  phi = (1'u - 1) / (1'v),  w = u - phi v,
// and the kriging variance is C(0) - w'c0 - phi (= w' gamma0 + mu with
// mu = -phi in the variogram form).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "krig_internal.h"

// Covariance C(h) = C(0) - gamma(h) at squared lag h2, written so that no
// cancellation occurs for h > 0.  Spherical: sill (1 - 1.5 q + 0.5 q^3) for
// q = h/a < 1, else 0.  Exponential (practical range): sill exp(-3h/a).
__device__ __forceinline__ double krig_cov(const krig_variogram& v, double h2)
{
    if (h2 == 0.0) return v.nugget + v.sill;
    double h = sqrt(h2);
    if (v.model == KRIG_SPHERICAL) {
        if (h >= v.range) return 0.0;
        double q = h / v.range;
        return v.sill * (1.0 - 1.5 * q + 0.5 * q * q * q);
    }
    return v.sill * exp(-3.0 * h / v.range);
}

// Lag tables of one volume.
//   gC[s][ay][ax], s in {0,1} (same / other known slice, dz = s*g),
//      ay, ax in [0, 2r]: covariance between two neighbourhood points.
//   g0[t-1][s][ay][ax], ay, ax in [0, r]: covariance between a point of the
//      lower (s=0, dz = t) or upper (s=1, dz = g-t) slice and the target.
struct LagDims {
    int r, g, n2r, nr;  // n2r = 2r+1, nr = r+1
    __device__ __forceinline__ int nC() const { return 2 * n2r * n2r; }
    __device__ __forceinline__ int n0() const { return (g - 1) * 2 * nr * nr; }
    __device__ __forceinline__ int iC(int s, int ay, int ax) const { return (s * n2r + ay) * n2r + ax; }
    __device__ __forceinline__ int i0(int t, int s, int ay, int ax) const
    {
        return (((t - 1) * 2 + s) * nr + ay) * nr + ax;
    }
};

__device__ __forceinline__ void krig_fill_lags(const LagDims& d, const krig_variogram& v, double* gC, double* g0,
                                               int tid, int nthreads)
{
    int nC = d.nC(), n0 = d.n0();
    for (int e = tid; e < nC + n0; e += nthreads) {
        if (e < nC) {
            int ax = e % d.n2r, ay = (e / d.n2r) % d.n2r, s = e / (d.n2r * d.n2r);
            double dz = (double)(s * d.g);
            gC[e] = krig_cov(v, (double)(ax * ax + ay * ay) + dz * dz);
        } else {
            int f = e - nC;
            int ax = f % d.nr, ay = (f / d.nr) % d.nr, s = (f / (d.nr * d.nr)) % 2, t = f / (2 * d.nr * d.nr) + 1;
            double dz = (double)(s == 0 ? t : d.g - t);
            g0[f] = krig_cov(v, (double)(ax * ax + ay * ay) + dz * dz);
        }
    }
}

// One neighbourhood point: offsets from the target pixel and its slice.
struct Tap {
    int8_t dx, dy, s, pad;
};

__device__ __forceinline__ double krig_cij(const LagDims& d, const double* gC, Tap a, Tap b)
{
    int ax = abs(a.dx - b.dx), ay = abs(a.dy - b.dy), s = a.s != b.s;
    return gC[d.iC(s, ay, ax)];
}

// Shared-memory workspace of one solve: up to KM points, NC <= LDX
// right-hand sides (NC-1 targets t plus the vector of ones).
template <typename TF, int KM, int LDX>
struct SolveSmem {
    TF L[KM * (KM + 1)];   // Cholesky factor, row-major, leading dimension K+1
    TF X[KM * LDX];        // right-hand sides / solutions in TF
    TF dinv[KM];           // 1 / L_kk
    double Xd[KM * LDX];   // solutions in FP64
    double Bd[KM * LDX];   // right-hand sides in FP64
    Tap tap[KM];
    int flag;
};

// Cholesky factorisation L L' = C (lower, in place) by one warp; lane i owns
// rows i, i+32.  Returns false (uniformly over the warp) if a pivot is not
// positive.
template <typename TF>
__device__ bool warp_cholesky(TF* L, TF* dinv, int K, int lane)
{
    const int ld = K + 1;
    for (int k = 0; k < K; ++k) {
        __syncwarp();
        TF d = L[k * ld + k];
        if (!(d > TF(0))) return false;
        TF l = sqrt(d);
        TF il = TF(1) / l;
        for (int i = k + 1 + lane; i < K; i += 32) L[i * ld + k] *= il;
        __syncwarp();
        if (lane == 0) {
            L[k * ld + k] = l;
            dinv[k] = il;
        }
        for (int i = k + 1 + lane; i < K; i += 32) {
            TF lik = L[i * ld + k];
            for (int j = k + 1; j <= i; ++j) L[i * ld + j] -= lik * L[j * ld + k];
        }
    }
    __syncwarp();
    return true;
}

// Solve L L' X = X in place for NC columns (leading dimension LDX), one warp.
template <typename TF, int LDX>
__device__ void warp_chol_solve(const TF* L, const TF* dinv, TF* X, int K, int NC, int lane)
{
    const int ld = K + 1;
    for (int k = 0; k < K; ++k) {  // forward: L y = b
        __syncwarp();
        if (lane < NC) X[k * LDX + lane] *= dinv[k];
        __syncwarp();
        for (int i = k + 1 + lane; i < K; i += 32) {
            TF lik = L[i * ld + k];
            for (int c = 0; c < NC; ++c) X[i * LDX + c] -= lik * X[k * LDX + c];
        }
    }
    for (int k = K - 1; k >= 0; --k) {  // backward: L' x = y
        __syncwarp();
        if (lane < NC) X[k * LDX + lane] *= dinv[k];
        __syncwarp();
        for (int i = lane; i < k; i += 32) {
            TF lki = L[k * ld + i];
            for (int c = 0; c < NC; ++c) X[i * LDX + c] -= lki * X[k * LDX + c];
        }
    }
    __syncwarp();
}

// Team-wide barrier: one warp (TEAM == 32) or the whole block.
template <int TEAM>
__device__ __forceinline__ void team_sync()
{
    if (TEAM == 32) __syncwarp();
    else __syncthreads();
}

// Solve the K-point ordinary-kriging systems whose taps are in S.tap and whose
// FP64 right-hand sides (c0 for each of NC-1 targets, then ones) are in S.Bd.
// C is built from the lag table gC.  TF = double: FP64 factorisation and
// solve.  TF = float: FP32 factorisation and solve followed by one FP64
// iterative-refinement step (residual B - C X in FP64, correction solved with
// the FP32 factor).  On return S.Xd holds u (columns 0..NC-2) and v (column
// NC-1) in FP64; the caller forms w = u - phi v.  Factorisation and
// triangular solves run on the team's first warp; build and residual on the
// whole team.  Returns false if C was not positive definite.
template <typename TF, int KM, int LDX, int TEAM>
__device__ bool team_ok_solve(SolveSmem<TF, KM, LDX>& S, const LagDims& d, const double* gC, int K, int NC, int tid)
{
    const int ld = K + 1;
    const int warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < K * K; e += TEAM) {
        int i = e / K, j = e % K;
        if (j <= i) S.L[i * ld + j] = (TF)krig_cij(d, gC, S.tap[i], S.tap[j]);
    }
    for (int e = tid; e < K * NC; e += TEAM) {
        int i = e / NC, c = e % NC;
        S.X[i * LDX + c] = (TF)S.Bd[i * LDX + c];
    }
    team_sync<TEAM>();
    if (warp == 0) {
        bool ok = warp_cholesky<TF>(S.L, S.dinv, K, lane);
        if (lane == 0) S.flag = ok ? 1 : 0;
        if (ok) warp_chol_solve<TF, LDX>(S.L, S.dinv, S.X, K, NC, lane);
    }
    team_sync<TEAM>();
    if (!S.flag) return false;
    for (int e = tid; e < K * NC; e += TEAM) {
        int i = e / NC, c = e % NC;
        S.Xd[i * LDX + c] = (double)S.X[i * LDX + c];
    }
    if (sizeof(TF) == 4) {
        team_sync<TEAM>();
        for (int e = tid; e < K * NC; e += TEAM) {
            int i = e / NC, c = e % NC;
            double s = S.Bd[i * LDX + c];
            Tap ti = S.tap[i];
            for (int j = 0; j < K; ++j) s -= krig_cij(d, gC, ti, S.tap[j]) * S.Xd[j * LDX + c];
            S.X[i * LDX + c] = (TF)s;
        }
        team_sync<TEAM>();
        if (warp == 0) warp_chol_solve<TF, LDX>(S.L, S.dinv, S.X, K, NC, lane);
        team_sync<TEAM>();
        for (int e = tid; e < K * NC; e += TEAM) {
            int i = e / NC, c = e % NC;
            S.Xd[i * LDX + c] += (double)S.X[i * LDX + c];
        }
    }
    team_sync<TEAM>();
    return true;
}

// Truncation slot of pixel coordinate p in [0, N): with l = min(p, r) and
// rr = min(N-1-p, r), the window covers p-l .. p+rr; slot = l*(r+1) + rr.
__device__ __forceinline__ int krig_slot(int p, int N, int r)
{
    int l = min(p, r), rr = min(N - 1 - p, r);
    return l * (r + 1) + rr;
}

__device__ __forceinline__ void krig_set_status(uint32_t* st, uint32_t bits)
{
    if (st) atomicOr(st, bits);
}

__device__ __forceinline__ int krig_find_vol(const KrigLaunch& P, int64_t idx, int which)
{
    int v = 0;
    for (int u = 1; u < P.n_vols; ++u) {
        int64_t b = which == 0 ? P.vol[u].item_begin : which == 1 ? P.vol[u].cls_begin : P.vol[u].vox_begin;
        if (b <= idx) v = u;
    }
    return v;
}
