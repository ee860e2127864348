// krig_ds_solve.cu -- class solve of the deduplicated-stencil (DS) form.
//
// A missing voxel's kriging system depends only on its geometry: its offset t
// inside the gap and how its (2r+1)^2 window is truncated at the in-plane
// border (Sec. 4.1.2: the system is built from distances between the target
// and its neighbouring known voxels; Appendix A: the weights solve the
// extended covariance system).  k_ds_solve solves each truncation class once,
// for every t at once, and writes the class's row of the weight table that
// k_ds_apply (krig_ds.cu) applies as a stencil.
#include <cuda_runtime.h>
#include <stdint.h>

#include "krig_device.cuh"

// ---------------------------------------------------------------------------
// Class solve: one block of 256 threads per xy-class.
// ---------------------------------------------------------------------------

// Combine u (columns 0..NC-2) and v (column NC-1) into the weights, phi and
// the kriging variance of each target t, and write the class's row of the
// weight and variance tables.
__device__ void ds_write_class(const KrigLaunch& P, const KrigVol& V, int cy, int cx, bool ok, const double* Xd,
                               const double* Bd, const Tap* tap, int K, int NC, double c00, double* phi,
                               double* vout)
{
    const int tid = threadIdx.x;
    const int lx = V.xext[cx][0], rx = V.xext[cx][1], ly = V.yext[cy][0], ry = V.yext[cy][1];
    const int nx = lx + rx + 1, ny = ly + ry + 1;
    // one warp per target column c: phi_c = (1'u_c - 1) / (1'v),
    // var_c = C(0) - w_c'c0_c - phi_c (the warps run concurrently)
    const int warp = tid >> 5, lane = tid & 31;
    if (ok && warp < NC - 1) {
        const int c = warp;
        double sv = 0.0, su = 0.0;
        for (int i = lane; i < K; i += 32) {
            sv += Xd[i * 8 + NC - 1];
            su += Xd[i * 8 + c];
        }
        for (int o = 16; o; o >>= 1) {
            sv += __shfl_xor_sync(0xffffffffu, sv, o);
            su += __shfl_xor_sync(0xffffffffu, su, o);
        }
        const double ph = (su - 1.0) / sv;
        double wc = 0.0;
        for (int i = lane; i < K; i += 32) wc += (Xd[i * 8 + c] - ph * Xd[i * 8 + NC - 1]) * Bd[i * 8 + c];
        for (int o = 16; o; o >>= 1) wc += __shfl_xor_sync(0xffffffffu, wc, o);
        if (lane == 0) {
            phi[c] = ph;
            vout[c] = c00 - wc - ph;
        }
    }
    __syncthreads();
    // Weight table row of this class: [s][dy+r][dx+r][t slot], zeros on
    // truncated taps and unused t slots.  u16 input: weights carry the scale.
    const int r = V.r;
    const int n2r = 2 * r + 1;
    const int ntap = 2 * n2r * n2r;
    const double scale = V.dtype == KRIG_U16 ? (double)V.scale : 1.0;
    const int64_t row = ((int64_t)cy * V.ncx + cx) * ntap * KRIG_TSLOTS;
    for (int e = tid; e < ntap * KRIG_TSLOTS; e += blockDim.x) {
        const int c = e % KRIG_TSLOTS, f = e / KRIG_TSLOTS;
        const int dx = f % n2r - r, dy = (f / n2r) % n2r - r, s = f / (n2r * n2r);
        double w = 0.0;
        if (c < NC - 1 && dx >= -lx && dx <= rx && dy >= -ly && dy <= ry) {
            const int i = (s * ny + (dy + ly)) * nx + (dx + lx);
            w = ok ? (Xd[i * 8 + c] - phi[c] * Xd[i * 8 + NC - 1]) * scale : __longlong_as_double(0x7ff8000000000000LL);
        }
        if (V.dtype == KRIG_F64) ((double*)(P.ws + V.wtab_off))[row + e] = w;
        else ((float*)(P.ws + V.wtab_off))[row + e] = (float)w;
    }
    // The interior class (full window) is invariant under the in-plane
    // symmetries of the square (D4), so its weights are constant on each orbit
    // {(dx, dy)} with the same (max, min) of |dx|, |dy|.  The stencil applies it
    // to orbit sums; the orbit weight is the mean over the orbit's members.
    if (cy * V.ncx + cx == V.cint) {
        for (int e = tid; e < 2 * KRIG_NORB * KRIG_TSLOTS; e += blockDim.x) {
            const int c = e % KRIG_TSLOTS, o = (e / KRIG_TSLOTS) % KRIG_NORB, s = e / (KRIG_TSLOTS * KRIG_NORB);
            double sum = 0.0;
            int cnt = 0;
            if (c < NC - 1) {
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx) {
                        const int a = max(abs(dx), abs(dy)), b = min(abs(dx), abs(dy));
                        if (a * (a + 1) / 2 + b != o) continue;
                        const int i = (s * ny + (dy + ly)) * nx + (dx + lx);
                        sum += ok ? (Xd[i * 8 + c] - phi[c] * Xd[i * 8 + NC - 1]) : __longlong_as_double(0x7ff8000000000000LL);
                        ++cnt;
                    }
            }
            const double w = cnt ? sum / cnt * scale : 0.0;
            if (V.dtype == KRIG_F64) ((double*)(P.ws + V.otab_off))[e] = w;
            else ((float*)(P.ws + V.otab_off))[e] = (float)w;
        }
    }
    if (tid < KRIG_TSLOTS) {
        float* vt = (float*)(P.ws + V.vtab_off) + ((int64_t)cy * V.ncx + cx) * KRIG_TSLOTS;
        vt[tid] = (tid < NC - 1) ? (ok ? (float)vout[tid] : __int_as_float(0x7fc00000)) : 0.0f;
    }
    (void)tap;
}

// Taps of class (cy, cx) in compact order (s, dy, dx) and the FP64
// right-hand sides: c0 of each target t = 1..g-1, then ones.
__device__ __forceinline__ int ds_class_setup(const KrigVol& V, const LagDims& d, const double* g0, int cy, int cx,
                                              Tap* tap, double* Bd)
{
    const int tid = threadIdx.x;
    const int lx = V.xext[cx][0], rx = V.xext[cx][1], ly = V.yext[cy][0], ry = V.yext[cy][1];
    const int nx = lx + rx + 1, ny = ly + ry + 1;
    const int K = 2 * nx * ny;
    const int NC = V.g;
    for (int i = tid; i < K; i += blockDim.x) {
        Tap tp;
        tp.s = (int8_t)(i / (nx * ny));
        tp.dy = (int8_t)((i / nx) % ny - ly);
        tp.dx = (int8_t)(i % nx - lx);
        tp.pad = 0;
        tap[i] = tp;
        for (int c = 0; c < NC; ++c)
            Bd[i * 8 + c] = c < NC - 1 ? g0[d.i0(c + 1, tp.s, abs((int)tp.dy), abs((int)tp.dx))] : 1.0;
    }
    __syncthreads();
    return K;
}

// ---------------------------------------------------------------------------
// Class solve by the Z-mirror split (FP32 factorisation, FP64 refinement).
//
// Both known slices carry the same in-plane window, so with the points
// ordered (lower slice, upper slice) the covariance matrix is C = [A B; B A]:
// A between points of one slice (dz = 0), B across the gap (dz = g), both
// symmetric.  x = [x0; x1] solves C x = [b0; b1] iff s = x0 + x1 and
// d = x0 - x1 solve (A + B) s = b0 + b1 and (A - B) d = b0 - b1, two SPD
// systems of n = nx * ny points each (C is SPD and the map is orthogonal up
// to a factor).  The ones vector gives b0 = b1 = 1 (d = 0); target t gives
// b0 = c_t, b1 = c_{g-t} (covariances to the lower / upper slice), so the sum
// system needs t = 1..floor(g/2) plus ones and the difference system
// t = 1..floor((g-1)/2); the other targets are the same columns mirrored.
// Ordinary kriging (Appendix A, one constant predictor) then gives
// u = C^-1 c0, v = C^-1 1, phi = (1'u - 1) / (1'v), w = u - phi v and the
// kriging variance C(0) - w'c0 - phi.
// ---------------------------------------------------------------------------
// distinct lags: (a >= b) pairs in [0, 2r] for dz = 0 and g, in [0, r] for dz = 1..g-1
constexpr int ZEV = (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 2) + (KRIG_GMAX - 1) * (KRIG_RMAX + 1) * (KRIG_RMAX + 2) / 2;

union DsSolveSmem {
    SolveSmem<double, KRIG_KMAX, 8> f64;
    ZSmem z;
};

// (a, b), a >= b >= 0, from its index a (a + 1) / 2 + b.
__device__ __forceinline__ void ds_pair(int idx, int* a, int* b)
{
    int q = 0;
    while ((q + 1) * (q + 2) / 2 <= idx) ++q;
    *a = q;
    *b = idx - q * (q + 1) / 2;
}

// Lag tables gC and g0 (same layout as krig_fill_lags) with one covariance
// evaluation per distinct lag: the in-plane part of a lag depends only on
// (max, min) of |dx|, |dy|, and the upper-slice target lags (dz = g - t)
// repeat the lower-slice ones (dz = t).
__device__ __forceinline__ int ds_lag_h2(const LagDims& d, int e, int nCp, int n0p)
{
    int a, b, dz;
    if (e < 2 * nCp) {
        ds_pair(e % nCp, &a, &b);
        dz = (e / nCp) * d.g;
    } else {
        const int f = e - 2 * nCp;
        ds_pair(f % n0p, &a, &b);
        dz = f / n0p + 1;
    }
    return a * a + b * b + dz * dz;
}
__device__ void ds_eval_lags(const LagDims& d, const krig_variogram& v, double* ev, int tid, int nt)
{
    const int nCp = d.n2r * (d.n2r + 1) / 2, n0p = d.nr * (d.nr + 1) / 2;
    const int ne = 2 * nCp + (d.g - 1) * n0p;
    for (int e = tid; e < ne; e += nt) ev[e] = krig_cov(v, (double)ds_lag_h2(d, e, nCp, n0p));
    __syncthreads();
}
// The same values as float-float pairs (the FP32 class solve).
__device__ void ds_eval_lags_ff(const LagDims& d, const krig_variogram& v, ff* ev, int tid, int nt)
{
    const int nCp = d.n2r * (d.n2r + 1) / 2, n0p = d.nr * (d.nr + 1) / 2;
    const int ne = 2 * nCp + (d.g - 1) * n0p;
    for (int e = tid; e < ne; e += nt) ev[e] = ff_from_double(krig_cov(v, (double)ds_lag_h2(d, e, nCp, n0p)));
    __syncthreads();
}
// Covariances from the distinct-lag table: between two points of the window
// (slice s = same / other, in-plane offsets ay, ax in [0, 2r]) and between a
// point (slice s, offsets in [0, r]) and target t.
template <typename E>
struct DsLags {
    const E* ev;
    int nCp, n0p, g;
    __device__ __forceinline__ DsLags(const LagDims& d, const E* e)
        : ev(e), nCp(d.n2r * (d.n2r + 1) / 2), n0p(d.nr * (d.nr + 1) / 2), g(d.g) {}
    __device__ __forceinline__ static int pair(int ay, int ax)
    {
        const int a = max(ax, ay), b = min(ax, ay);
        return a * (a + 1) / 2 + b;
    }
    __device__ __forceinline__ E c(int s, int ay, int ax) const { return ev[s * nCp + pair(ay, ax)]; }
    __device__ __forceinline__ E c0(int t, int s, int ay, int ax) const
    {
        const int dz = s == 0 ? t : g - t;
        return ev[2 * nCp + (dz - 1) * n0p + pair(ay, ax)];
    }
};
// The same values expanded into the lag tables gC, g0 (layout of krig_fill_lags).
__device__ void ds_fill_lags(const LagDims& d, const krig_variogram& v, double* gC, double* g0, double* ev, int tid,
                             int nt)
{
    ds_eval_lags(d, v, ev, tid, nt);
    const int nCp = d.n2r * (d.n2r + 1) / 2, n0p = d.nr * (d.nr + 1) / 2;
    const int nC = d.nC(), n0 = d.n0();
    for (int e = tid; e < nC + n0; e += nt) {
        if (e < nC) {
            const int ax = e % d.n2r, ay = (e / d.n2r) % d.n2r, s = e / (d.n2r * d.n2r);
            const int a = max(ax, ay), b = min(ax, ay);
            gC[e] = ev[s * nCp + a * (a + 1) / 2 + b];
        } else {
            const int f = e - nC;
            const int ax = f % d.nr, ay = (f / d.nr) % d.nr, s = (f / (d.nr * d.nr)) % 2, t = f / (2 * d.nr * d.nr) + 1;
            const int a = max(ax, ay), b = min(ax, ay), dz = s == 0 ? t : d.g - t;
            g0[f] = ev[2 * nCp + (dz - 1) * n0p + a * (a + 1) / 2 + b];
        }
    }
    __syncthreads();
}
// One weight-table entry: FP64 volumes take the pair's value, FP32 volumes its
// nearest float, u16 volumes the weight times the intensity scale (rounded once).
__device__ __forceinline__ void ds_store_weight(const KrigVol& V, float* tf, double* td, int64_t i, ff w)
{
    if (V.dtype == KRIG_F64) td[i] = ff_to_double(w);
    else if (V.dtype == KRIG_U16) tf[i] = ff_round(ff_mul_f(w, V.scale));
    else tf[i] = ff_round(w);
}
// Solve, combine and write one truncation class: FP32 factorisation, the
// residual, the combine and the tables in float-float.
template <int NT>
__device__ void ds_class_zsplit(const KrigLaunch& P, const KrigVol& V, int cy, int cx, const DsLags<ff>& lg, ZSmem& S,
                                int tid)
{
    const int warp = tid >> 5, lane = tid & 31;
    const int lx = V.xext[cx][0], rx = V.xext[cx][1], ly = V.yext[cy][0], ry = V.yext[cy][1];
    const int nx = lx + rx + 1, ny = ly + ry + 1, n = nx * ny;
    const int g = V.g, r = V.r, n2r = 2 * r + 1;
    const int hp = g / 2, hm = (g - 1) / 2;  // sum / difference targets
    const int m0 = 1 + hp, m1 = hm;  // columns of the sum / difference system
    // system entries by lag, points, right-hand sides
    for (int e = tid; e < n2r * n2r; e += NT) {
        const ff a = lg.c(0, e / n2r, e % n2r), b = lg.c(1, e / n2r, e % n2r);
        S.T[0][e] = ff_add(a, b);
        S.T[1][e] = ff_sub(a, b);
    }
    for (int e = tid; e < ZL; e += NT) {
        S.dx[e] = (int8_t)(e < n ? e % nx - lx : 0);
        S.dy[e] = (int8_t)(e < n ? e / nx - ly : 0);
    }
    for (int e = tid; e < n * 8; e += NT) {
        const int i = e >> 3, c = e & 7;
        const int ax = abs(i % nx - lx), ay = abs(i / nx - ly);
        ff bp = ff_make(0.0f), bm = ff_make(0.0f);
        if (c == 0) bp = ff_make(2.0f);
        else if (c <= hp) bp = ff_add(lg.c0(c, 0, ay, ax), lg.c0(c, 1, ay, ax));
        if (c < hm) bm = ff_sub(lg.c0(c + 1, 0, ay, ax), lg.c0(c + 1, 1, ay, ax));
        S.B[0][i][c] = bp;
        S.B[1][i][c] = bm;
    }
    if (tid == 0) S.fail = 0;
    __syncthreads();
    const int msys[2] = {m0, m1};
    ds_fill_rows(S, m1 > 0 ? 2 : 1, n, msys, n2r, tid, NT);
    __syncthreads();
    // FP32 factorisation: the sum system on warp 0, the difference system on warp 1
    if (warp < 2 && (warp == 0 || m1 > 0)) {
        if (!ds_warp_gj(S, warp, n, lane) && lane == 0) S.fail = 1;
    }
    __syncthreads();
    const bool ok = !S.fail;
    // refinement: R = B - S X (compensated), X += S^-1 R in FP32, X kept as a pair
    const int nv = n * (m0 + m1);  // (system, point, column) triples
    if (ok) {
        // one (system, point, column) per thread: nv <= ZN * 8 <= NT
        const int z = tid < n * m0 ? 0 : 1, f = z ? tid - n * m0 : tid, m = z ? m1 : m0;
        const int i = m ? f / m : 0, c = m ? f % m : 0;
        if (tid < nv) {
            const int dxi = S.dx[i], dyi = S.dy[i];
            ff_dot acc(S.B[z][i][c]);
            for (int j = 0; j < n; ++j)
                acc.add(S.T[z][abs(dyi - S.dy[j]) * n2r + abs(dxi - S.dx[j])], -S.M[z][j][c]);
            S.R[z][i][c] = ff_round(acc.value());
        }
        __syncthreads();
        if (tid < nv) {
            const float* ai = &S.M[z][i][ZL - n];  // row i of S^-1
            float corr = 0.0f;
            for (int j = 0; j < n; ++j) corr = fmaf(ai[j], S.R[z][j][c], corr);
            S.X[z][i][c] = ff_two_sum(S.M[z][i][c], corr);
        }
        __syncthreads();
        // combine, one warp per target t (lane = point):
        //   sum column p = min(t, g-t), difference column p-1 with sign +1 for
        //   t < g-t, -1 for t > g-t, none for t = g/2
        if (warp < g - 1) {
            const int t = warp + 1, p = min(t, g - t);
            const bool in = lane < n;
            const ff zero = ff_make(0.0f);
            const ff sv = in ? S.X[0][lane][0] : zero, st = in ? S.X[0][lane][p] : zero;
            ff sd = zero;
            if (in && t != g - t) sd = t < g - t ? S.X[1][lane][p - 1] : ff_neg(S.X[1][lane][p - 1]);
            const ff a = ff_warp_sum(sv), b = ff_warp_sum(st);
            const ff ph = ff_div(ff_sub(b, ff_make(1.0f)), a);
            const ff hv = ff_scale2(ff_mul(ph, sv), 0.5f);
            const ff w0 = ff_sub(ff_scale2(ff_add(st, sd), 0.5f), hv), w1 = ff_sub(ff_scale2(ff_sub(st, sd), 0.5f), hv);
            ff wc = zero;
            if (in) {
                const int ax = abs(S.dx[lane]), ay = abs(S.dy[lane]);
                wc = ff_add(ff_mul(w0, lg.c0(t, 0, ay, ax)), ff_mul(w1, lg.c0(t, 1, ay, ax)));
                S.W[0][lane][t - 1] = w0;
                S.W[1][lane][t - 1] = w1;
            }
            wc = ff_warp_sum(wc);
            if (lane == 0) S.var[t - 1] = ff_round(ff_sub(ff_sub(lg.c(0, 0, 0), wc), ph));
        }
        __syncthreads();
    } else if (tid == 0) {
        krig_set_status(P.status, KRIG_DEV_SINGULAR);
    }
    // weight-table row of the class: [s][dy+r][dx+r][t slot], zeros on
    // truncated taps and unused t slots; u16 input: weights carry the scale
    const int n2 = n2r * n2r, ntap = 2 * n2;
    const int64_t row = ((int64_t)cy * V.ncx + cx) * ntap * KRIG_TSLOTS;
    for (int e = tid; e < ntap * KRIG_TSLOTS; e += NT) {
        const int c = e % KRIG_TSLOTS, f = e / KRIG_TSLOTS;
        const int dx = f % n2r - r, dy = (f / n2r) % n2r - r, s = f / n2;
        ff w = ff_make(0.0f);
        if (c < g - 1 && dx >= -lx && dx <= rx && dy >= -ly && dy <= ry)
            w = ok ? S.W[s][(dy + ly) * nx + dx + lx][c] : ff_make(__int_as_float(0x7fc00000));
        ds_store_weight(V, (float*)(P.ws + V.wtab_off), (double*)(P.ws + V.wtab_off), row + e, w);
    }
    // interior class: weight per D4 orbit.  The class is D4-symmetric, so the
    // members of an orbit carry the same weight up to rounding; the table takes
    // the member (dx, dy) = (a, b) of orbit (a, b), a >= b >= 0.
    if (cy * V.ncx + cx == V.cint) {
        for (int e = tid; e < 2 * KRIG_NORB * KRIG_TSLOTS; e += NT) {
            const int c = e % KRIG_TSLOTS, o = (e / KRIG_TSLOTS) % KRIG_NORB, s = e / (KRIG_TSLOTS * KRIG_NORB);
            ff w = ff_make(0.0f);
            if (c < g - 1 && o < (r + 1) * (r + 2) / 2) {
                int oa, ob;
                ds_pair(o, &oa, &ob);
                w = ok ? S.W[s][(ob + ly) * nx + oa + lx][c] : ff_make(__int_as_float(0x7fc00000));
            }
            ds_store_weight(V, (float*)(P.ws + V.otab_off), (double*)(P.ws + V.otab_off), e, w);
        }
    }
    if (tid < KRIG_TSLOTS) {
        float* vt = (float*)(P.ws + V.vtab_off) + ((int64_t)cy * V.ncx + cx) * KRIG_TSLOTS;
        vt[tid] = (tid < g - 1) ? (ok ? S.var[tid] : __int_as_float(0x7fc00000)) : 0.0f;
    }
}
template <typename TF>
__global__ void __launch_bounds__(256) k_ds_solve(const __grid_constant__ KrigLaunch P)
{
    __shared__ DsSolveSmem U;
    __shared__ double gC[2 * (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1)];
    __shared__ double g0[(KRIG_GMAX - 1) * 2 * (KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    __shared__ double phi[8], vout[8];
    __shared__ __align__(8) unsigned char evb[ZEV * 8];  // distinct-lag covariances: double or pair

    const int tid = threadIdx.x;
    // the stencil's frame-unit tickets start from zero (it reads them after this grid completes)
    if (blockIdx.x == 0 && tid < 3) ((unsigned*)(P.ws + KRIG_CTRL_FRAME_NEXT))[tid] = 0u;
    // let the stencil kernel launch now; it waits for this grid before it reads the tables
    asm volatile("griddepcontrol.launch_dependents;");
    const int64_t cls = blockIdx.x;
    const int v = krig_find_vol(P, cls, 1);
    const KrigVol& V = P.vol[v];
    if (V.g < 2) return;  // no missing slices: nothing to solve
    const int local = (int)(cls - V.cls_begin);
    const int cy = local / V.ncx, cx = local % V.ncx;
    const krig_variogram vg = P.vg[v];
    const int r = V.r;
    LagDims d{r, V.g, 2 * r + 1, r + 1};
    if (sizeof(TF) == 8) {
        ds_fill_lags(d, vg, gC, g0, (double*)evb, tid, 256);
        SolveSmem<double, KRIG_KMAX, 8>& S = U.f64;
        const int K = ds_class_setup(V, d, g0, cy, cx, S.tap, S.Bd);
        const bool ok = team_ok_solve<double, KRIG_KMAX, 8, 256>(S, d, gC, K, V.g, tid);
        if (!ok && tid == 0) krig_set_status(P.status, KRIG_DEV_SINGULAR);
        ds_write_class(P, V, cy, cx, ok, S.Xd, S.Bd, S.tap, K, V.g, gC[0], phi, vout);
    } else {
        ds_eval_lags_ff(d, vg, (ff*)evb, tid, 256);
        ds_class_zsplit<256>(P, V, cy, cx, DsLags<ff>(d, (const ff*)evb), U.z, tid);
    }
}

int krig_launch_ds_solve(const KrigLaunch& L, int solve_fp64, void* stream)
{
    if (L.n_classes == 0) return 0;
    dim3 grid((unsigned)L.n_classes);
    if (solve_fp64) k_ds_solve<double><<<grid, 256, 0, (cudaStream_t)stream>>>(L);
    else k_ds_solve<float><<<grid, 256, 0, (cudaStream_t)stream>>>(L);
    return (int)cudaGetLastError();
}

