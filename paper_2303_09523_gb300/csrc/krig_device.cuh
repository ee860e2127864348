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

#include <type_traits>

#include "krig_internal.h"
#include "krig_ff.cuh"

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

// ---------------------------------------------------------------------------
// Register-resident FP32 factorisation for one warp.
//
// Lane l holds rows i = l + 32q (q < ROWS) of the KM x KM matrix in a[q][*];
// rows and columns past the system size K are identity, so the leading K x K
// block factors exactly as if alone.  Right-looking Cholesky: at step k the
// pivot and column k are broadcast with warp shuffles, and each lane updates
// its own rows.  All loop bounds are compile-time, so the matrix never leaves
// registers.  Returns false (warp-uniform) if a pivot is not positive.
// ---------------------------------------------------------------------------
template <int KM>
struct RegDim {
    static constexpr int ROWS = (KM + 31) / 32;
    static constexpr int LDL = KM + 1;  // odd leading dimension of L in shared memory
};

// Compile-time loop: calls f(integral_constant<int, i>) for i in [B, E).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

template <int KM, typename T = float>
__device__ __forceinline__ bool warp_chol_reg(T (&a)[RegDim<KM>::ROWS][KM], int lane)
{
    constexpr int ROWS = RegDim<KM>::ROWS;
    bool ok = true;
    static_for<0, KM>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const T piv = __shfl_sync(0xffffffffu, a[k / 32][k], k % 32);
        ok = ok && (piv > T(0));
        const T l = sqrt(piv);
        const T il = T(1) / l;
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const int i = lane + 32 * q;
            if (i > k) a[q][k] *= il;
            else if (i == k) a[q][k] = l;
        }
        static_for<k + 1, KM>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const T ljk = __shfl_sync(0xffffffffu, a[j / 32][k], j % 32);
#pragma unroll
            for (int q = 0; q < ROWS; ++q) {
                const int i = lane + 32 * q;
                if (i >= j) a[q][j] = fma(-a[q][k], ljk, a[q][j]);
            }
        });
    });
    return ok;
}

// Store the factor (lower triangle, row-major, leading dimension KM+1) and the
// reciprocal diagonal to shared memory.
template <int KM, typename T = float>
__device__ __forceinline__ void warp_store_factor(const T (&a)[RegDim<KM>::ROWS][KM], T* Ls, T* dinv, int lane)
{
    constexpr int ROWS = RegDim<KM>::ROWS, LDL = RegDim<KM>::LDL;
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
        const int i = lane + 32 * q;
        if (i < KM) {
#pragma unroll
            for (int j = 0; j < KM; ++j)
                if (j <= i) Ls[i * LDL + j] = a[q][j];
#pragma unroll
            for (int j = 0; j < KM; ++j)
                if (j == i) dinv[i] = T(1) / a[q][j];
        }
    }
}

// Solve L L' x = x for one right-hand side held by the warp (lane l owns
// x[q] = x_{l+32q}), with L and 1/diag(L) in shared memory.
template <int KM, typename T = float>
__device__ __forceinline__ void warp_sweep(const T* Ls, const T* dinv, T (&x)[RegDim<KM>::ROWS], int lane)
{
    constexpr int ROWS = RegDim<KM>::ROWS, LDL = RegDim<KM>::LDL;
    static_for<0, KM>([&](auto kc) {  // forward: L y = b
        constexpr int k = decltype(kc)::value;
        const T xk = __shfl_sync(0xffffffffu, x[k / 32], k % 32) * dinv[k];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const int i = lane + 32 * q;
            if (i == k) x[q] = xk;
            else if (i > k && i < KM) x[q] = fma(-Ls[i * LDL + k], xk, x[q]);
        }
    });
    static_for<0, KM>([&](auto kc) {  // backward: L' x = y
        constexpr int k = KM - 1 - decltype(kc)::value;
        const T xk = __shfl_sync(0xffffffffu, x[k / 32], k % 32) * dinv[k];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const int i = lane + 32 * q;
            if (i == k) x[q] = xk;
            else if (i < k) x[q] = fma(-Ls[k * LDL + i], xk, x[q]);
        }
    });
}

// Per-warp shared memory of a per-voxel solve (two right-hand sides: c0 and ones).
template <int KM, typename T>
struct VoxSmem {
    T Ls[KM * (KM + 1)];
    T dinv[KM];
    double Bd[KM * 2];
    double Xd[KM * 2];
    Tap tap[KM];
};

// One warp solves one voxel's system with the register factorisation.
// T = double: FP64 factorisation and sweeps (no refinement).  T = float:
// FP32 factorisation and sweeps plus one FP64 refinement step (the residual
// B - C X is formed in FP64 from the FP64 lag table).  On return S.Xd holds
// u (column 0) and v (column 1) in FP64.
template <int KM, typename T>
__device__ bool warp_ok_solve_vox(VoxSmem<KM, T>& S, const LagDims& d, const double* gC, int K, int lane)
{
    constexpr int ROWS = RegDim<KM>::ROWS;
    T a[ROWS][KM];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
        const int i = lane + 32 * q;
        const Tap ti = S.tap[i < K ? i : 0];
#pragma unroll
        for (int j = 0; j < KM; ++j) {
            T v;
            if (i < K && j < K) v = (T)krig_cij(d, gC, ti, S.tap[j]);
            else v = (i == j) ? T(1) : T(0);
            a[q][j] = v;
        }
    }
    const bool ok = warp_chol_reg<KM, T>(a, lane);
    if (!ok) return false;
    warp_store_factor<KM, T>(a, S.Ls, S.dinv, lane);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        T x[ROWS];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const int i = lane + 32 * q;
            x[q] = i < K ? (T)S.Bd[i * 2 + c] : T(0);
        }
        warp_sweep<KM, T>(S.Ls, S.dinv, x, lane);
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const int i = lane + 32 * q;
            if (i < K) S.Xd[i * 2 + c] = (double)x[q];
        }
    }
    __syncwarp();
    if (sizeof(T) == 4) {
        T rres[2][ROWS];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const int i = lane + 32 * q;
            double s0 = 0.0, s1 = 0.0;
            if (i < K) {
                s0 = S.Bd[i * 2 + 0];
                s1 = S.Bd[i * 2 + 1];
                const Tap ti = S.tap[i];
                for (int j = 0; j < K; ++j) {
                    const double cij = krig_cij(d, gC, ti, S.tap[j]);
                    s0 -= cij * S.Xd[j * 2 + 0];
                    s1 -= cij * S.Xd[j * 2 + 1];
                }
            }
            rres[0][q] = (T)s0;
            rres[1][q] = (T)s1;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            warp_sweep<KM, T>(S.Ls, S.dinv, rres[c], lane);
#pragma unroll
            for (int q = 0; q < ROWS; ++q) {
                const int i = lane + 32 * q;
                if (i < K) S.Xd[i * 2 + c] += (double)rres[c][q];
            }
        }
        __syncwarp();
    }
    return true;
}

// ---------------------------------------------------------------------------
// Half-size SPD systems of the Z-mirror split (class solves of the DS form
// and of the leave-one-slice-out loss): in-plane points of the window only.
// ---------------------------------------------------------------------------
constexpr int ZN = (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1);  // in-plane points, <= 25
constexpr int ZL = 32;                                         // register row: n + m <= 25 + 5
static_assert(ZN + 1 + KRIG_GMAX / 2 <= ZL, "register row too short");
static_assert(ZN * 8 <= 256, "one refinement entry per thread");

constexpr int ZLP = ZL + 4;  // padded row of the augmented matrices: float4-aligned, rows 4 banks apart

struct ZSmem {
    ff T[2][ZN];              // A + B, A - B entries by in-plane lag ay * (2r+1) + ax
    ff B[2][ZN][8];           // right-hand sides
    ff X[2][ZN][8];           // refined solutions
    float R[2][ZN][8];        // residuals rounded to FP32
    ff W[2][ZN][8];           // weights: [slice][point][t-1]
    float var[8];             // kriging variance per target
    // [S | B] rows before the factorisation, [X | 0 | S^-1] after (each row
    // divided by its pivot): X at columns 0..m-1, S^-1 at ZL-n..ZL-1
    __align__(16) float M[2][ZN][ZLP];
    __align__(16) float row[2][2][ZL];  // pivot-row broadcast, [system][step parity]
    int8_t dx[ZL], dy[ZL];
    int fail;
};

// Row i of the augmented system z in FP32: the system entries (from the lag
// table T), then the m right-hand sides, then zeros.  All threads of the block
// fill the rows (e over 2 * ZN * ZL) before the factorisation.
__device__ __forceinline__ void ds_fill_rows(ZSmem& S, int nsys, int n, const int* msys, int n2r, int tid, int nt)
{
    for (int e = tid; e < nsys * n * ZL; e += nt) {
        const int j = e % ZL, i = (e / ZL) % n, z = e / (ZL * n);
        float a = 0.0f;
        if (j < n) a = S.T[z][abs(S.dy[i] - S.dy[j]) * n2r + abs(S.dx[i] - S.dx[j])].hi;
        else if (j < n + msys[z]) a = S.B[z][i][j - n].hi;
        S.M[z][i][j] = a;
    }
}

// Gauss-Jordan on the rows of S.M[z] by one warp, lane i holding row i in
// registers.  Each step drops the pivot column from the front of every row and
// appends the identity column it turns into, so that every register index is
// static: after n steps a row holds [X | 0 | S^-1] (up to the row's pivot,
// divided out at the end), stored back in place.  The pivot row reaches the
// other lanes through shared memory (one buffer per step parity: a step's
// stores cannot overtake the previous step's reads).  No pivoting (S is SPD);
// a pivot that is not positive fails.
__device__ __forceinline__ bool ds_warp_gj(ZSmem& S, int z, int n, int lane)
{
    float r[ZL];
    const float4* src = reinterpret_cast<const float4*>(S.M[z][lane < n ? lane : 0]);
#pragma unroll
    for (int q = 0; q < ZL / 4; ++q) {
        const float4 v = lane < n ? src[q] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        r[4 * q] = v.x;
        r[4 * q + 1] = v.y;
        r[4 * q + 2] = v.z;
        r[4 * q + 3] = v.w;
    }
    float dk = 1.0f;
    bool ok = true;
    for (int k = 0; k < n; ++k) {
        float4* buf = reinterpret_cast<float4*>(S.row[z][k & 1]);
        if (lane == k) {
#pragma unroll
            for (int q = 0; q < ZL / 4; ++q) buf[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        }
        __syncwarp();
        const float4 v0 = buf[0];
        const float p0 = v0.x;
        if (!(p0 > 0.0f)) {  // the same value in every lane
            ok = false;
            break;
        }
        const bool piv = lane == k;
        const float fi = r[0] * __frcp_rn(p0);
        const float f = piv ? 0.0f : fi;
        if (piv) dk = p0;
        r[0] = fmaf(-f, v0.y, r[1]);
        r[1] = fmaf(-f, v0.z, r[2]);
        r[2] = fmaf(-f, v0.w, r[3]);
#pragma unroll
        for (int q = 1; q < ZL / 4; ++q) {
            const float4 v = buf[q];
            r[4 * q - 1] = fmaf(-f, v.x, r[4 * q]);
            r[4 * q] = fmaf(-f, v.y, r[4 * q + 1]);
            r[4 * q + 1] = fmaf(-f, v.z, r[4 * q + 2]);
            r[4 * q + 2] = fmaf(-f, v.w, r[4 * q + 3]);
        }
        r[ZL - 1] = piv ? 1.0f : -fi;
    }
    if (ok && lane < n) {
        const float di = 1.0f / dk;
        float4* dst = reinterpret_cast<float4*>(S.M[z][lane]);
#pragma unroll
        for (int q = 0; q < ZL / 4; ++q)
            dst[q] = make_float4(r[4 * q] * di, r[4 * q + 1] * di, r[4 * q + 2] * di, r[4 * q + 3] * di);
    }
    return ok;
}

// ---------------------------------------------------------------------------
// Packed pixel pairs: one quantity at two adjacent pixels as one value (FP32: a
// 64-bit register pair and the f32x2 instructions, each half rounding as the
// scalar instruction; FP64: two doubles).  Stencils over D4 orbit sums use them
// so that their arithmetic needs no operand shuffling.
// ---------------------------------------------------------------------------
// Two floats as one 64-bit register pair and back (operands of the packed
// f32x2 instructions).
__device__ __forceinline__ unsigned long long pk2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}


// One quantity at two adjacent pixels.
template <typename TC> struct Px2;
template <> struct Px2<float> {
    unsigned long long v;
    __device__ __forceinline__ static Px2 of(float a, float b) { return {pk2(a, b)}; }
    __device__ __forceinline__ static Px2 zero() { return {0ull}; }
    __device__ __forceinline__ float x() const { float a, b; upk2(v, a, b); return a; }
    __device__ __forceinline__ float y() const { float a, b; upk2(v, a, b); return b; }
};
template <> struct Px2<double> {
    double a, b;
    __device__ __forceinline__ static Px2 of(double x, double y) { return {x, y}; }
    __device__ __forceinline__ static Px2 zero() { return {0.0, 0.0}; }
    __device__ __forceinline__ double x() const { return a; }
    __device__ __forceinline__ double y() const { return b; }
};
__device__ __forceinline__ Px2<float> operator+(Px2<float> p, Px2<float> q)
{
    Px2<float> r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(p.v), "l"(q.v));
    return r;
}
__device__ __forceinline__ Px2<double> operator+(Px2<double> p, Px2<double> q) { return {p.a + q.a, p.b + q.b}; }
// acc += w * z, half by half
__device__ __forceinline__ void px_fma(Px2<float>& acc, Px2<float> w, Px2<float> z)
{
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc.v) : "l"(w.v), "l"(z.v));
}
__device__ __forceinline__ void px_fma(Px2<double>& acc, Px2<double> w, Px2<double> z)
{
    acc.a = fma(w.a, z.a, acc.a);
    acc.b = fma(w.b, z.b, acc.b);
}
// A weight of the shared-memory table as the pair (w, w): FP32 tables hold the
// pair already, FP64 tables the value.
__device__ __forceinline__ Px2<float> px_w(unsigned long long w) { return {w}; }
__device__ __forceinline__ Px2<double> px_w(double w) { return {w, w}; }

// Pixel pair k (columns m = 4 + 2k, m + 1) of a row of pairs: the values
// themselves, c[m - 1] + c[m + 1] (shift 1) and c[m - 2] + c[m + 2] (shift 2).
template <typename TC>
__device__ __forceinline__ Px2<TC> px_s1(const Px2<TC> (&c)[6], int k)
{
    const int h = 2 + k;  // pair index of column m
    return Px2<TC>::of(c[h - 1].y() + c[h].y(), c[h].x() + c[h + 1].x());
}
template <typename TC>
__device__ __forceinline__ Px2<TC> px_s2(const Px2<TC> (&c)[6], int k)
{
    return c[1 + k] + c[3 + k];
}
