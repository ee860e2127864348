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

union DsSolveSmem {
    SolveSmem<double, KRIG_KMAX, 8> f64;
    GJSmem gj;
};

template <typename TF>
__global__ void __launch_bounds__(256) k_ds_solve(const __grid_constant__ KrigLaunch P)
{
    __shared__ DsSolveSmem U;
    __shared__ double gC[2 * (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1)];
    __shared__ double g0[(KRIG_GMAX - 1) * 2 * (KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    __shared__ double phi[8], vout[8];

    const int tid = threadIdx.x;
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
    krig_fill_lags(d, vg, gC, g0, tid, 256);
    __syncthreads();
    if (sizeof(TF) == 8) {
        SolveSmem<double, KRIG_KMAX, 8>& S = U.f64;
        const int K = ds_class_setup(V, d, g0, cy, cx, S.tap, S.Bd);
        const bool ok = team_ok_solve<double, KRIG_KMAX, 8, 256>(S, d, gC, K, V.g, tid);
        if (!ok && tid == 0) krig_set_status(P.status, KRIG_DEV_SINGULAR);
        ds_write_class(P, V, cy, cx, ok, S.Xd, S.Bd, S.tap, K, V.g, gC[0], phi, vout);
    } else {
        GJSmem& S = U.gj;
        const int K = ds_class_setup(V, d, g0, cy, cx, S.tap, S.Bd);
        const bool ok = block_gj_solve<256>(S, d, gC, K, V.g, tid);
        if (!ok && tid == 0) krig_set_status(P.status, KRIG_DEV_SINGULAR);
        ds_write_class(P, V, cy, cx, ok, S.Xd, S.Bd, S.tap, K, V.g, gC[0], phi, vout);
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

