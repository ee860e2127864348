// krig_loo.cu -- leave-one-slice-out (LOO) cross-validation loss of the
// kriging interpolator and its adjoint, for fitting the variogram by gradient.
//
// The paper fixes no variogram (Sec. 4.1.2, Appendix A give only the kriging
// system).  LOO turns the interpolator into a loss: each interior known slice
// j (1..n-2) is predicted at its own z from slices j-1 and j+1, which sit g
// below and above it -- the interpolation geometry with a gap of 2g at t = g --
// by the same ordinary kriging (Appendix A, one constant predictor):
//     P_j(x,y) = sum_k w_{c(x,y),k} S_{j+-1}(x+dx_k, y+dy_k),
//     r_j = P_j - S_j,   L = 1/((n-2) H W) sum_j sum_{x,y} r_j^2.
// Gradients (for an upstream gL = dOut/dL):
//   dL/dS_m(p) = 2gL/N [ sum_d r_{m+1}(p-d) w_{c(p-d)}(lower, d)
//                        + sum_d r_{m-1}(p-d) w_{c(p-d)}(upper, d) - r_m(p) ]
//   dL/dw_{c,k} = 2gL/N sum_{voxels of class c} r S_k
//   dL/dtheta: adjoint of the bordered solve A lambda = b (A symmetric):
//     A abar = [wbar; 0],  dL/dtheta_p = abar_w' (dc0/dtheta_p - dC/dtheta_p w).
// The class systems are re-solved in the backward pass rather than stored.
#include <cuda_runtime.h>
#include <stdint.h>

#include "krig_device.cuh"

#define LOO_TX 64
#define LOO_TY 16
#define LOO_PAD 4
#define LOO_RP (LOO_TX + 2 * LOO_PAD)

// dC/d(nugget, sill, range) at squared lag h2 (C(h) = nugget + sill - gamma(h)).
__device__ __forceinline__ void krig_cov_grad(const krig_variogram& v, double h2, double d[3])
{
    if (h2 == 0.0) {
        d[0] = 1.0;
        d[1] = 1.0;
        d[2] = 0.0;
        return;
    }
    const double h = sqrt(h2), a = v.range;
    d[0] = 0.0;
    if (v.model == KRIG_SPHERICAL) {
        if (h >= a) {
            d[1] = 0.0;
            d[2] = 0.0;
        } else {
            const double q = h / a;
            d[1] = 1.0 - 1.5 * q + 0.5 * q * q * q;
            d[2] = v.sill * (1.5 * h / (a * a) - 1.5 * h * h * h / (a * a * a * a));
        }
    } else {
        const double e = exp(-3.0 * h / a);
        d[1] = e;
        d[2] = v.sill * e * 3.0 * h / (a * a);
    }
}

// ---------------------------------------------------------------------------
// Class kernel: one block per (volume, xy-class).  mode 0: LOO weights.
// mode 1: weights and the adjoint contribution of this class to dL/dtheta.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_loo_class(const __grid_constant__ KrigLaunch P, int mode)
{
    __shared__ GJSmem S;
    __shared__ double gC[2 * (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1)];
    __shared__ double g0[2 * (KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    __shared__ double dC[3][2 * (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1)];
    __shared__ double d0[3][2 * (KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    __shared__ double wgt[KRIG_KMAX], abar[KRIG_KMAX], red[8][4];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int v = 0;
    for (int u = 1; u < P.n_vols; ++u)
        if (P.vol[u].loo_cls_begin <= blockIdx.x) v = u;
    const KrigVol& V = P.vol[v];
    const int local = (int)(blockIdx.x - V.loo_cls_begin);
    const int cy = local / V.ncx, cx = local % V.ncx;
    const krig_variogram vg = P.vg[v];
    const int r = V.r, n2r = 2 * r + 1, nr = r + 1;
    const int g2 = 2 * V.g;  // LOO: bracketing slices 2g apart, target in the middle
    LagDims d{r, g2, n2r, nr};
    const int nC = 2 * n2r * n2r, n0 = 2 * nr * nr;
    for (int e = tid; e < nC + n0; e += 256) {
        double h2, dd[3];
        if (e < nC) {
            const int ax = e % n2r, ay = (e / n2r) % n2r, s = e / (n2r * n2r);
            h2 = (double)(ax * ax + ay * ay) + (double)(s * g2) * (double)(s * g2);
            gC[e] = krig_cov(vg, h2);
            krig_cov_grad(vg, h2, dd);
            for (int p = 0; p < 3; ++p) dC[p][e] = dd[p];
        } else {
            const int f = e - nC;
            const int ax = f % nr, ay = (f / nr) % nr;
            h2 = (double)(ax * ax + ay * ay) + (double)V.g * (double)V.g;  // dz = g both sides
            g0[f] = krig_cov(vg, h2);
            krig_cov_grad(vg, h2, dd);
            for (int p = 0; p < 3; ++p) d0[p][f] = dd[p];
        }
    }
    __syncthreads();
    const int lx = V.xext[cx][0], rx = V.xext[cx][1], ly = V.yext[cy][0], ry = V.yext[cy][1];
    const int nx = lx + rx + 1, ny = ly + ry + 1;
    const int K = 2 * nx * ny;
    const int NC = mode == 0 ? 2 : 3;  // c0, ones, [wbar]
    const double* lbar = (const double*)(P.ws + V.lbar_off) + (int64_t)local * (2 * n2r * n2r);
    const double coef = mode == 0 ? 0.0 : 2.0 * P.grad_loss[v] / ((double)(V.n - 2) * V.H * V.W);
    for (int i = tid; i < K; i += 256) {
        Tap tp;
        tp.s = (int8_t)(i / (nx * ny));
        tp.dy = (int8_t)((i / nx) % ny - ly);
        tp.dx = (int8_t)(i % nx - lx);
        tp.pad = 0;
        S.tap[i] = tp;
        S.Bd[i * 8 + 0] = g0[(tp.s * nr + abs((int)tp.dy)) * nr + abs((int)tp.dx)];
        S.Bd[i * 8 + 1] = 1.0;
        if (mode == 1) {
            const int full = (tp.s * n2r + (tp.dy + r)) * n2r + (tp.dx + r);
            S.Bd[i * 8 + 2] = coef * lbar[full];  // wbar = 2 gL / N * sum r S_k
        }
    }
    __syncthreads();
    const bool ok = block_gj_solve<256>(S, d, gC, K, NC, tid);
    if (!ok) {
        if (tid == 0) krig_set_status(P.status, KRIG_DEV_SINGULAR);
        return;
    }
    // sums over the taps: 1'u, 1'v, 1'x
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = tid; i < K; i += 256) {
        s0 += S.Xd[i * 8 + 0];
        s1 += S.Xd[i * 8 + 1];
        if (mode == 1) s2 += S.Xd[i * 8 + 2];
    }
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        red[warp][0] = s0;
        red[warp][1] = s1;
        red[warp][2] = s2;
    }
    __syncthreads();
    double su = 0.0, sv = 0.0, sx = 0.0;
    for (int w = 0; w < 8; ++w) {
        su += red[w][0];
        sv += red[w][1];
        sx += red[w][2];
    }
    const double phi = (su - 1.0) / sv;
    const double aphi = sx / sv;
    for (int i = tid; i < K; i += 256) {
        wgt[i] = S.Xd[i * 8 + 0] - phi * S.Xd[i * 8 + 1];
        if (mode == 1) abar[i] = S.Xd[i * 8 + 2] - aphi * S.Xd[i * 8 + 1];
    }
    __syncthreads();
    if (mode == 0) {
        // LOO weight row in the full tap layout [s][dy+r][dx+r], zeros on truncated taps
        float* lw = (float*)(P.ws + V.lw_off) + (int64_t)local * (2 * n2r * n2r);
        for (int f = tid; f < 2 * n2r * n2r; f += 256) {
            const int dx = f % n2r - r, dy = (f / n2r) % n2r - r, s = f / (n2r * n2r);
            float w = 0.0f;
            if (dx >= -lx && dx <= rx && dy >= -ly && dy <= ry) w = (float)wgt[(s * ny + (dy + ly)) * nx + (dx + lx)];
            lw[f] = w;
        }
        return;
    }
    // dL/dtheta_p = abar' (dc0/dtheta_p - dC/dtheta_p w), one term per (i, p)
    double tp3[3] = {0.0, 0.0, 0.0};
    for (int i = tid; i < K; i += 256) {
        const Tap ti = S.tap[i];
        const int i0 = (ti.s * nr + abs((int)ti.dy)) * nr + abs((int)ti.dx);
        double acc[3] = {d0[0][i0], d0[1][i0], d0[2][i0]};
        for (int j = 0; j < K; ++j) {
            const Tap tj = S.tap[j];
            const int ic = d.iC(ti.s != tj.s, abs(ti.dy - tj.dy), abs(ti.dx - tj.dx));
            for (int p = 0; p < 3; ++p) acc[p] -= dC[p][ic] * wgt[j];
        }
        for (int p = 0; p < 3; ++p) tp3[p] += abar[i] * acc[p];
    }
    for (int p = 0; p < 3; ++p)
        for (int o = 16; o; o >>= 1) tp3[p] += __shfl_xor_sync(0xffffffffu, tp3[p], o);
    __syncthreads();
    if (lane == 0)
        for (int p = 0; p < 3; ++p) red[warp][p] = tp3[p];
    __syncthreads();
    if (tid < 3) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][tid];
        atomicAdd(P.grad_params + 3 * v + tid, s);
    }
}

// ---------------------------------------------------------------------------
// Residual kernel: one block per (volume, target slice j, 64 x 16 tile).
// mode 0: loss (and optional prediction).  mode 1: loss, residual buffer and
// the per-class tap sums sum r S_k for dL/dw.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float loo_load(const void* in, int dtype, float scale, size_t idx)
{
    if (dtype == KRIG_F32) return ((const float*)in)[idx];
    if (dtype == KRIG_U16) return __fmul_rn((float)((const uint16_t*)in)[idx], scale);
    return (float)((const double*)in)[idx];
}

template <int R>
__device__ void loo_residual_tile(const KrigLaunch& P, int v, int j, int x0, int y0, int mode, float* sm)
{
    constexpr int N2R = 2 * R + 1, NTAP = 2 * N2R * N2R;
    constexpr int ROWS = LOO_TY + 2 * R;
    const KrigVol& V = P.vol[v];
    const int H = V.H, W = V.W;
    const size_t plane = (size_t)H * W;
    float* lo = sm;
    float* hi = sm + ROWS * LOO_RP;
    float* ce = hi + ROWS * LOO_RP;                  // LOO_TY x LOO_TX, target slice
    float* sg = ce + LOO_TY * LOO_TX;                // [ncls][NTAP] tap sums (mode 1)
    double* sl = (double*)(sg + 32 * NTAP + 2);      // loss partials of the warps (8)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncls = V.ncx * V.ncy;
    for (int e = tid; e < ROWS * LOO_RP; e += 256) {
        const int rr = e / LOO_RP, cc = e % LOO_RP;
        const int yy = y0 - R + rr, xx = x0 - LOO_PAD + cc;
        float a = 0.f, b = 0.f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
            a = loo_load(P.in[v], V.dtype, V.scale, (size_t)(j - 1) * plane + (size_t)yy * W + xx);
            b = loo_load(P.in[v], V.dtype, V.scale, (size_t)(j + 1) * plane + (size_t)yy * W + xx);
        }
        lo[e] = a;
        hi[e] = b;
    }
    for (int e = tid; e < LOO_TY * LOO_TX; e += 256) {
        const int yy = y0 + e / LOO_TX, xx = x0 + e % LOO_TX;
        ce[e] = (yy < H && xx < W) ? loo_load(P.in[v], V.dtype, V.scale, (size_t)j * plane + (size_t)yy * W + xx) : 0.f;
    }
    if (mode == 1)
        for (int e = tid; e < ncls * NTAP; e += 256) sg[e] = 0.f;
    __syncthreads();
    const int lrow = (warp >> 2) * 8 + (lane >> 2);
    const int lcol = (warp & 3) * 16 + (lane & 3) * 4;
    const int y = y0 + lrow;
    const float* lw = (const float*)(P.ws + V.lw_off);
    float gi[NTAP];
#pragma unroll
    for (int k = 0; k < NTAP; ++k) gi[k] = 0.f;
    double loss = 0.0;
    if (y < H) {
        const int cy = V.ymap[krig_slot(y, H, R)];
        for (int p = 0; p < 4; ++p) {
            const int x = x0 + lcol + p;
            if (x >= W) break;
            const int c = cy * V.ncx + V.xmap[krig_slot(x, W, R)];
            const float* wr = lw + (int64_t)c * NTAP;
            float pred = 0.f;
            float taps[NTAP];
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int dy = -R; dy <= R; ++dy)
#pragma unroll
                    for (int dx = -R; dx <= R; ++dx) {
                        const int k = (s * N2R + (dy + R)) * N2R + (dx + R);
                        const float z = (s == 0 ? lo : hi)[(lrow + R + dy) * LOO_RP + LOO_PAD + lcol + p + dx];
                        taps[k] = z;
                        pred = fmaf(__ldg(wr + k), z, pred);
                    }
            const float res = pred - ce[lrow * LOO_TX + lcol + p];
            loss += (double)res * (double)res;
            const size_t oidx = (size_t)(j - 1) * plane + (size_t)y * W + x;
            if (mode == 0) {
                if (P.pred[v]) P.pred[v][oidx] = pred;
            } else {
                ((float*)(P.ws + V.res_off))[oidx] = res;
                if (c == V.cint) {
#pragma unroll
                    for (int k = 0; k < NTAP; ++k) gi[k] = fmaf(res, taps[k], gi[k]);
                } else {
#pragma unroll
                    for (int k = 0; k < NTAP; ++k) atomicAdd(&sg[c * NTAP + k], res * taps[k]);
                }
            }
        }
    }
    // loss: warp -> block -> volume accumulator
    for (int o = 16; o; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) sl[warp] = loss;
    if (mode == 1 && V.cint >= 0) {
#pragma unroll
        for (int k = 0; k < NTAP; ++k) {
            float t = gi[k];
            for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) atomicAdd(&sg[V.cint * NTAP + k], t);
        }
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sl[w];
        atomicAdd((double*)(P.ws + V.lacc_off), s);
    }
    if (mode == 1) {
        double* lbar = (double*)(P.ws + V.lbar_off);
        for (int e = tid; e < ncls * NTAP; e += 256)
            if (sg[e] != 0.f) atomicAdd(lbar + e, (double)sg[e]);
    }
}

__global__ void __launch_bounds__(256) k_loo_residual(const __grid_constant__ KrigLaunch P, int mode)
{
    extern __shared__ __align__(16) float lsm[];
    const int64_t it = blockIdx.x;
    int v = 0;
    for (int u = 1; u < P.n_vols; ++u)
        if (P.vol[u].loo_item_begin <= it) v = u;
    const KrigVol& V = P.vol[v];
    const int64_t local = it - V.loo_item_begin;
    const int tiles = V.tiles_x * V.tiles_y;
    const int j = 1 + (int)(local / tiles);
    const int tile = (int)(local % tiles);
    const int x0 = (tile % V.tiles_x) * LOO_TX, y0 = (tile / V.tiles_x) * LOO_TY;
    switch (V.r) {
    case 0: loo_residual_tile<0>(P, v, j, x0, y0, mode, lsm); break;
    case 1: loo_residual_tile<1>(P, v, j, x0, y0, mode, lsm); break;
    default: loo_residual_tile<2>(P, v, j, x0, y0, mode, lsm); break;
    }
}

// ---------------------------------------------------------------------------
// Adjoint w.r.t. the slices, gather form: one block per (volume, slice m, tile).
// ---------------------------------------------------------------------------
template <int R>
__device__ void loo_adjoint_tile(const KrigLaunch& P, int v, int m, int x0, int y0, float* sm)
{
    constexpr int N2R = 2 * R + 1, NTAP = 2 * N2R * N2R;
    constexpr int ROWS = LOO_TY + 2 * R;
    const KrigVol& V = P.vol[v];
    const int H = V.H, W = V.W, n = V.n;
    const size_t plane = (size_t)H * W;
    const float* res = (const float*)(P.ws + V.res_off);  // r_j at (j-1)
    float* rup = sm;                   // r_{m+1}: predictions for which S_m is the lower slice
    float* rdn = sm + ROWS * LOO_RP;   // r_{m-1}: predictions for which S_m is the upper slice
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool has_up = m + 1 <= n - 2, has_dn = m - 1 >= 1;
    for (int e = tid; e < ROWS * LOO_RP; e += 256) {
        const int rr = e / LOO_RP, cc = e % LOO_RP;
        const int yy = y0 - R + rr, xx = x0 - LOO_PAD + cc;
        float a = 0.f, b = 0.f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
            if (has_up) a = res[(size_t)m * plane + (size_t)yy * W + xx];        // r_{m+1} at index m
            if (has_dn) b = res[(size_t)(m - 2) * plane + (size_t)yy * W + xx];  // r_{m-1} at index m-2
        }
        rup[e] = a;
        rdn[e] = b;
    }
    __syncthreads();
    const int lrow = (warp >> 2) * 8 + (lane >> 2);
    const int lcol = (warp & 3) * 16 + (lane & 3) * 4;
    const int y = y0 + lrow;
    if (y >= H) return;
    const float* lw = (const float*)(P.ws + V.lw_off);
    const double coef = 2.0 * P.grad_loss[v] / ((double)(n - 2) * H * W);
    float* gs = P.grad_slices[v];
    for (int p = 0; p < 4; ++p) {
        const int x = x0 + lcol + p;
        if (x >= W) break;
        float acc = 0.f;
#pragma unroll
        for (int dy = -R; dy <= R; ++dy) {
            const int qy = y - dy;
            if (qy < 0 || qy >= H) continue;
            const int cyq = V.ymap[krig_slot(qy, H, R)];
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                const int qx = x - dx;
                if (qx < 0 || qx >= W) continue;
                const float* wr = lw + (int64_t)(cyq * V.ncx + V.xmap[krig_slot(qx, W, R)]) * NTAP;
                const int off = (lrow + R - dy) * LOO_RP + LOO_PAD + lcol + p - dx;
                acc = fmaf(__ldg(wr + (0 * N2R + (dy + R)) * N2R + (dx + R)), rup[off], acc);  // S_m lower of m+1
                acc = fmaf(__ldg(wr + (1 * N2R + (dy + R)) * N2R + (dx + R)), rdn[off], acc);  // S_m upper of m-1
            }
        }
        double gval = (double)acc;
        if (m >= 1 && m <= n - 2) gval -= (double)res[(size_t)(m - 1) * plane + (size_t)y * W + x];
        gval *= coef;
        const size_t oidx = (size_t)m * plane + (size_t)y * W + x;
        if (P.accumulate) gs[oidx] += (float)gval;
        else gs[oidx] = (float)gval;
    }
}

__global__ void __launch_bounds__(256) k_loo_adjoint(const __grid_constant__ KrigLaunch P)
{
    extern __shared__ __align__(16) float lsm[];
    const int64_t it = blockIdx.x;
    int v = 0;
    for (int u = 1; u < P.n_vols; ++u)
        if (P.vol[u].loo_adj_begin <= it) v = u;
    const KrigVol& V = P.vol[v];
    if (!P.grad_slices[v]) return;
    const int64_t local = it - V.loo_adj_begin;
    const int tiles = V.tiles_x * V.tiles_y;
    const int m = (int)(local / tiles);
    const int tile = (int)(local % tiles);
    const int x0 = (tile % V.tiles_x) * LOO_TX, y0 = (tile / V.tiles_x) * LOO_TY;
    switch (V.r) {
    case 0: loo_adjoint_tile<0>(P, v, m, x0, y0, lsm); break;
    case 1: loo_adjoint_tile<1>(P, v, m, x0, y0, lsm); break;
    default: loo_adjoint_tile<2>(P, v, m, x0, y0, lsm); break;
    }
}

__global__ void k_loo_finalize(const __grid_constant__ KrigLaunch P)
{
    const int v = threadIdx.x;
    if (v >= P.n_vols) return;
    const KrigVol& V = P.vol[v];
    P.loss[v] = *(const double*)(P.ws + V.lacc_off) / ((double)(V.n - 2) * V.H * V.W);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static size_t loo_smem(const KrigLaunch& L, int adjoint)
{
    size_t m = 0;
    for (int v = 0; v < L.n_vols; ++v) {
        const int r = L.vol[v].r;
        const int rows = LOO_TY + 2 * r;
        const int ntap = 2 * (2 * r + 1) * (2 * r + 1);
        size_t b = adjoint ? (size_t)2 * rows * LOO_RP * 4
                           : (size_t)2 * rows * LOO_RP * 4 + LOO_TY * LOO_TX * 4 + (32 * ntap + 2) * 4 + 8 * 8 + 16;
        if (b > m) m = b;
    }
    return m;
}

int krig_launch_loo(const KrigLaunch& L, int backward, int want_grad_slices, int want_grad_params, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    // zero the loss accumulators and (backward) the tap sums
    for (int v = 0; v < L.n_vols; ++v) {
        const KrigVol& V = L.vol[v];
        e = cudaMemsetAsync(L.ws + V.lacc_off, 0, sizeof(double), st);
        if (e != cudaSuccess) return (int)e;
        if (backward) {
            const size_t nb = (size_t)V.ncx * V.ncy * 2 * (2 * V.r + 1) * (2 * V.r + 1) * sizeof(double);
            e = cudaMemsetAsync(L.ws + V.lbar_off, 0, nb, st);
            if (e != cudaSuccess) return (int)e;
        }
    }
    k_loo_class<<<(unsigned)L.n_loo_classes, 256, 0, st>>>(L, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    const size_t s1 = loo_smem(L, 0);
    if (s1 > 48 * 1024) cudaFuncSetAttribute(k_loo_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1);
    k_loo_residual<<<(unsigned)L.n_loo_items, 256, s1, st>>>(L, backward ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    if (!backward) {
        k_loo_finalize<<<1, 64, 0, st>>>(L);
        return (int)cudaGetLastError();
    }
    if (want_grad_slices) {
        const size_t s2 = loo_smem(L, 1);
        k_loo_adjoint<<<(unsigned)L.n_loo_adj, 256, s2, st>>>(L);
        if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    }
    if (want_grad_params) {
        k_loo_class<<<(unsigned)L.n_loo_classes, 256, 0, st>>>(L, 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    }
    return 0;
}
