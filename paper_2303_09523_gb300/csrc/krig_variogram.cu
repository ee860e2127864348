// krig_variogram.cu -- method-of-moments empirical variogram of the known
// slices: the data a variogram model (Sec. 4.1.2 uses gamma(h) without saying
// how it is estimated) is fitted to.
//
// For every lag vector (s, dy, dx), |dy|, |dx| <= L, s = 0 (within one known
// slice) or 1 (known slice k to k + 1), the kernel sums (S[k, y, x] -
// S[k + s, y + dy, x + dx])^2 over all voxel pairs inside the stack.  One block
// per (known slice k, band of EV_TY rows) walks the band's 64-column tiles;
// each tile of slice k and of slice k + 1 is staged with a halo of L in shared
// memory, and each thread owns up to EV_OPT lag vectors, summing a row of at
// most 64 pixels in FP32 and everything above it in FP64.  The bound is the
// FP32 pipe (a subtract and a fused multiply-add per pair); HBM is read about
// (2 + 4L/EV_TY) times per slice through the halos.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "krig_internal.h"

#define EV_TX 64
#define EV_TY 16
#define EV_THREADS 512
#define EV_LMAX 16
#define EV_OPT ((2 * (2 * EV_LMAX + 1) * (2 * EV_LMAX + 1) + EV_THREADS - 1) / EV_THREADS)

__device__ __forceinline__ float ev_load(const void* in, int dtype, float scale, size_t idx)
{
    if (dtype == KRIG_F32) return ((const float*)in)[idx];
    if (dtype == KRIG_U16) return __fmul_rn((float)((const uint16_t*)in)[idx], scale);
    return (float)((const double*)in)[idx];
}

__global__ void __launch_bounds__(EV_THREADS) k_emp_variogram(const void* in, int dtype, float scale, int n, int H,
                                                               int W, int L, double* sums)
{
    extern __shared__ float ev_sm[];
    const int q = 2 * L + 1, SP = EV_TX + 2 * L, ROWS = EV_TY + 2 * L;
    float* t0 = ev_sm;              // slice k: rows y0-L .. y0+EV_TY+L-1, columns x0-L .. x0+EV_TX+L-1
    float* t1 = ev_sm + ROWS * SP;  // slice k+1, same window
    const int k = blockIdx.x, y0 = blockIdx.y * EV_TY;
    const bool up = k + 1 < n;
    const int nO = (up ? 2 : 1) * q * q;  // lag vectors this block contributes to
    const size_t plane = (size_t)H * W;
    const int ty = min(EV_TY, H - y0);
    double acc[EV_OPT];
#pragma unroll
    for (int j = 0; j < EV_OPT; ++j) acc[j] = 0.0;
    for (int x0 = 0; x0 < W; x0 += EV_TX) {
        __syncthreads();  // the previous tile's reads are done
        for (int e = threadIdx.x; e < ROWS * SP; e += EV_THREADS) {
            const int yy = y0 - L + e / SP, xx = x0 - L + e % SP;
            const bool inside = yy >= 0 && yy < H && xx >= 0 && xx < W;
            const size_t off = (size_t)yy * W + xx;
            t0[e] = inside ? ev_load(in, dtype, scale, (size_t)k * plane + off) : 0.f;
            if (up) t1[e] = inside ? ev_load(in, dtype, scale, (size_t)(k + 1) * plane + off) : 0.f;
        }
        __syncthreads();
        const int tx = min(EV_TX, W - x0);
#pragma unroll
        for (int j = 0; j < EV_OPT; ++j) {
            const int o = threadIdx.x + j * EV_THREADS;
            if (o < nO) {
                const int s = o / (q * q), rem = o - s * q * q, dy = rem / q - L, dx = rem % q - L;
                // tile pixels (yy, xx) whose partner (yy + dy, xx + dx) lies inside the slice
                const int ya = max(0, -dy - y0), yb = min(ty, H - dy - y0);
                const int xa = max(0, -dx - x0), xb = min(tx, W - dx - x0);
                const float* A = t0 + L * SP + L;
                const float* B = (s ? t1 : t0) + (L + dy) * SP + L + dx;
                double part = 0.0;
                for (int yy = ya; yy < yb; ++yy) {
                    float r = 0.f;
                    for (int xx = xa; xx < xb; ++xx) {
                        const float d = A[yy * SP + xx] - B[yy * SP + xx];
                        r = fmaf(d, d, r);
                    }
                    part += (double)r;
                }
                acc[j] += part;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < EV_OPT; ++j) {
        const int o = threadIdx.x + j * EV_THREADS;
        if (o < nO && acc[j] != 0.0) atomicAdd(sums + o, acc[j]);
    }
}

extern "C" krig_status krig_empirical_variogram(const krig_volume_desc* desc, const void* d_slices, int32_t max_lag,
                                                double* d_sums, int64_t* h_counts, void* stream)
{
    if (!desc || !d_slices || !d_sums) {
        krig_internal_set_error("desc, d_slices and d_sums must not be NULL");
        return KRIG_EINVAL;
    }
    const krig_volume_desc& d = *desc;
    if (d.H < 1 || d.H > 65536 || d.W < 1 || d.W > 65536 || d.n_known < 1 || d.n_known > 65536 ||
        (d.in_dtype != KRIG_F64 && d.in_dtype != KRIG_F32 && d.in_dtype != KRIG_U16) ||
        (d.in_dtype == KRIG_U16 && !(d.in_scale > 0.0f && d.in_scale < 3.0e38f))) {
        krig_internal_set_error("invalid volume descriptor (H, W, n_known, in_dtype, in_scale)");
        return KRIG_EINVAL;
    }
    if (max_lag < 0 || max_lag > EV_LMAX) {
        krig_internal_set_error("max_lag must be in [0, 16]");
        return KRIG_EINVAL;
    }
    const int L = max_lag, q = 2 * L + 1;
    if (h_counts) {
        // terms per lag vector: (n - s) slices x (H - |dy|) rows x (W - |dx|) columns
        for (int s = 0; s < 2; ++s)
            for (int dy = -L; dy <= L; ++dy)
                for (int dx = -L; dx <= L; ++dx) {
                    const int64_t ns = d.n_known - s, hy = d.H - (dy < 0 ? -dy : dy), wx = d.W - (dx < 0 ? -dx : dx);
                    h_counts[(s * q + dy + L) * q + dx + L] = (ns > 0 && hy > 0 && wx > 0) ? ns * hy * wx : 0;
                }
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_sums, 0, sizeof(double) * 2 * q * q, st);
    if (e == cudaSuccess) {
        const dim3 grid((unsigned)d.n_known, (unsigned)((d.H + EV_TY - 1) / EV_TY));
        const size_t smem = sizeof(float) * 2 * (EV_TY + 2 * L) * (EV_TX + 2 * L);
        k_emp_variogram<<<grid, EV_THREADS, smem, st>>>(d_slices, d.in_dtype, d.in_dtype == KRIG_U16 ? d.in_scale : 1.0f,
                                                        d.n_known, d.H, d.W, L, d_sums);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        krig_internal_set_error(cudaGetErrorString(e));
        return KRIG_ECUDA;
    }
    return KRIG_OK;
}
