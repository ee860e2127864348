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

#include <algorithm>

#include "krig_device.cuh"

#define LOO_TX 64
#define LOO_TY 16
#define LOO_PAD 4
#define LOO_RP (LOO_TX + 2 * LOO_PAD)
// Shared-memory row stride of the tiles: 80 floats puts two consecutive rows
// in opposite halves of the 32 banks, so the 16-byte loads of a quarter warp
// (two rows x four 4-pixel groups) hit 32 distinct banks.
#define LOO_SP 80

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

__device__ __forceinline__ bool loo_same_bits(double a, double b)
{
    return __double_as_longlong(a) == __double_as_longlong(b);
}

// ---------------------------------------------------------------------------
// Class kernel: one block per (volume, xy-class).  mode 0: LOO weights (and
// a record of the variogram they were solved for).  mode 2: the same, unless
// the record shows that the weights in the workspace already belong to this
// variogram (the backward pass after the forward pass of the same step).
// mode 1: weights and the adjoint contribution of this class to dL/dtheta.
//
// The two bracketing slices carry the same window and sit symmetrically
// (dz = -g, +g) about the target, so with C = [A B; B A] (B across dz = 2g)
// both right-hand sides c0 = [c; c] and 1 are symmetric: only the sum system
// (A + B) s = b0 + b1 is needed, and w0 = w1 = (s_u - phi s_v) / 2.  For
// dL/dtheta, sum_i abar_i (dc0_i - (dC w)_i) runs over both slices with equal
// brackets, so only abar_lower + abar_upper = s_x - (1's_x / 1's_v) s_v enters,
// with s_x from the same sum system at right-hand side wbar_lower + wbar_upper.
// Arithmetic: covariances in FP64, FP32 factorisation, residuals, combine and
// adjoint in float-float (this GPU's FP64 rate is 1/64 of FP32); the dL/dtheta
// sums leave in FP64.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_loo_class(const __grid_constant__ KrigLaunch P, int mode_in)
{
    __shared__ ZSmem S;
    __shared__ ff gC[2 * (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1)];
    __shared__ ff g0[(KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    __shared__ ff dC[3][2 * (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1)];
    __shared__ ff d0[3][(KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    __shared__ ff wgt[ZN], abar[ZN], red[8][4];
    __shared__ ff tsum[ZN], osum[KRIG_NORB];  // mode 1: tap and orbit sums over the copies
    __shared__ ff svs;                        // 1's_v
    static_assert(KRIG_LOO_REP == 32, "one copy per lane in the reductions below");

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // programmatic dependent launch: let the next kernel of the pass launch.  The
    // class solve itself reads only the variogram and the geometry, so it runs
    // before the wait for the previous kernel (overlapping its tail); everything
    // that touches the pass's accumulators, weights or record runs after the wait.
    asm volatile("griddepcontrol.launch_dependents;");
    int v = 0;
    for (int u = 1; u < P.n_vols; ++u)
        if (P.vol[u].loo_cls_begin <= blockIdx.x) v = u;
    const KrigVol& V = P.vol[v];
    const int local = (int)(blockIdx.x - V.loo_cls_begin);
    const int cy = local / V.ncx, cx = local % V.ncx;
    const krig_variogram vg = P.vg[v];
    const int ncls = V.ncx * V.ncy, taps = 2 * (2 * V.r + 1) * (2 * V.r + 1);
    // a new pass: zero the volume's loss sums and (backward) the dL/dw sums, spread
    // over its class blocks; the kernels that add to them run after this launch
    auto zero_pass = [&]() {
        for (int e = local * 256 + tid; e < KRIG_LOO_REP; e += ncls * 256) ((double*)(P.ws + V.lacc_off))[e] = 0.0;
        if (mode_in == 2) {
            for (int e = local * 256 + tid; e < KRIG_LOO_REP * ncls * taps; e += ncls * 256)
                ((double*)(P.ws + V.lbar_off))[e] = 0.0;
            for (int e = local * 256 + tid; e < KRIG_LOO_REP * KRIG_NORB; e += ncls * 256)
                ((double*)(P.ws + V.lorb_off))[e] = 0.0;
            if (P.grad_params && !P.accumulate && local == 0 && tid < 3) P.grad_params[3 * v + tid] = 0.0;
        }
    };
    krig_variogram* rec = (krig_variogram*)(P.ws + V.lvg_off);
    if (mode_in == 2) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        zero_pass();
        if (rec->model == vg.model && loo_same_bits(rec->nugget, vg.nugget) && loo_same_bits(rec->sill, vg.sill) &&
            loo_same_bits(rec->range, vg.range))
            return;  // these weights are already in the workspace
    }
    const int mode = mode_in == 1 ? 1 : 0;
    const int r = V.r, n2r = 2 * r + 1, nr = r + 1;
    const int g2 = 2 * V.g;  // LOO: bracketing slices 2g apart, target in the middle
    const int nC = 2 * n2r * n2r, n0 = nr * nr;
    // covariances (and, in the adjoint pass, their derivatives) in FP64, kept as pairs
    for (int e = tid; e < nC + n0; e += 256) {
        int h2;
        double dd[3];
        if (e < nC) {
            const int ax = e % n2r, ay = (e / n2r) % n2r, s = e / (n2r * n2r);
            h2 = ax * ax + ay * ay + (s * g2) * (s * g2);
            gC[e] = ff_from_double(krig_cov(vg, (double)h2));
            if (mode == 1) {
                krig_cov_grad(vg, (double)h2, dd);
#pragma unroll
                for (int p = 0; p < 3; ++p) dC[p][e] = ff_from_double(dd[p]);
            }
        } else {
            const int f = e - nC;
            const int ax = f % nr, ay = f / nr;
            h2 = ax * ax + ay * ay + V.g * V.g;  // dz = g both sides
            g0[f] = ff_from_double(krig_cov(vg, (double)h2));
            if (mode == 1) {
                krig_cov_grad(vg, (double)h2, dd);
#pragma unroll
                for (int p = 0; p < 3; ++p) d0[p][f] = ff_from_double(dd[p]);
            }
        }
    }
    __syncthreads();
    const int lx = V.xext[cx][0], rx = V.xext[cx][1], ly = V.yext[cy][0], ry = V.yext[cy][1];
    const int nx = lx + rx + 1, ny = ly + ry + 1;
    const int n = nx * ny;  // in-plane points (per slice)
    const int nn = n2r * n2r;
    for (int e = tid; e < nn; e += 256) S.T[0][e] = ff_add(gC[e], gC[nn + e]);  // A + B at in-plane lag e
    for (int e = tid; e < ZL; e += 256) {
        S.dx[e] = (int8_t)(e < n ? e % nx - lx : 0);
        S.dy[e] = (int8_t)(e < n ? e / nx - ly : 0);
    }
    // right-hand sides 2c and 2 (ones); the adjoint's third one (wbar) comes after the wait
    for (int i = tid; i < n; i += 256) {
        const int dx = i % nx - lx, dy = i / nx - ly;
        S.B[0][i][0] = ff_scale2(g0[abs(dy) * nr + abs(dx)], 2.0f);
        S.B[0][i][1] = ff_make(2.0f);
    }
    if (tid == 0) S.fail = 0;
    __syncthreads();
    const int msys[2] = {2, 0};
    ds_fill_rows(S, 1, n, msys, n2r, tid, 256);
    __syncthreads();
    if (warp == 0 && !ds_warp_gj(S, 0, n, lane) && lane == 0) S.fail = 1;
    __syncthreads();
    if (S.fail) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        if (mode_in == 0) zero_pass();
        if (tid == 0) krig_set_status(P.status, KRIG_DEV_SINGULAR);
        return;
    }
    // refinement of columns c0..c0+m-1 (threads i * m + c): R = B - (A+B) X
    // compensated, X += (A+B)^-1 R in FP32, X kept as a pair
    auto refine = [&](int c0, int m) {
        const int nv = n * m;
        const int i = tid / m, c = c0 + tid % m;
        if (tid < nv) {
            ff_dot acc(S.B[0][i][c]);
            for (int j = 0; j < n; ++j)
                acc.add(S.T[0][abs(S.dy[i] - S.dy[j]) * n2r + abs(S.dx[i] - S.dx[j])], -S.M[0][j][c]);
            S.R[0][i][c] = ff_round(acc.value());
        }
        __syncthreads();
        if (tid < nv) {
            const float* ai = &S.M[0][i][ZL - n];  // row i of (A+B)^-1
            float corr = 0.0f;
            for (int j = 0; j < n; ++j) corr = fmaf(ai[j], S.R[0][j][c], corr);
            S.X[0][i][c] = ff_two_sum(S.M[0][i][c], corr);
        }
        __syncthreads();
    };
    refine(0, 2);
    // sums over the points (one warp: n <= 32): 1's_u, 1's_v; phi and the weights
    if (warp == 0) {
        const ff zero = ff_make(0.0f);
        const ff xu = lane < n ? S.X[0][lane][0] : zero, xv = lane < n ? S.X[0][lane][1] : zero;
        const ff su = ff_warp_sum(xu), sv = ff_warp_sum(xv);
        const ff phi = ff_div(ff_sub(su, ff_make(1.0f)), sv);
        if (lane < n) wgt[lane] = ff_scale2(ff_sub(xu, ff_mul(phi, xv)), 0.5f);
        if (lane == 0) svs = sv;
    }
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous kernel of the pass is complete
    if (mode_in == 0) zero_pass();
    if (mode == 0) {
        // LOO weight row in the full tap layout [s][dy+r][dx+r] (the same in both
        // slices), zeros on truncated taps
        float* lw = (float*)(P.ws + V.lw_off) + (int64_t)local * (2 * nn);
        for (int f = tid; f < 2 * nn; f += 256) {
            const int dx = f % n2r - r, dy = (f / n2r) % n2r - r;
            float w = 0.0f;
            if (dx >= -lx && dx <= rx && dy >= -ly && dy <= ry) w = ff_round(wgt[(dy + ly) * nx + (dx + lx)]);
            lw[f] = w;
        }
        if (local == V.cint && tid < (r + 1) * (r + 2) / 2) {
            // interior class: weight per D4 orbit (mean over the orbit's taps of one
            // slice), stored after the weight table for the stencil kernels
            float sum = 0.f;
            int cnt = 0;
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    const int qa = max(abs(dx), abs(dy)), qb = min(abs(dx), abs(dy));
                    if (qa * (qa + 1) / 2 + qb == tid) {
                        sum += ff_round(wgt[(dy + r) * n2r + (dx + r)]);
                        ++cnt;
                    }
                }
            ((float*)(P.ws + V.lw_off))[loo_wo_off(V.ncx * V.ncy * 2 * nn) + tid] = sum / (float)cnt;
        }
        if (tid == 0) *rec = vg;  // read by a later launch only
        return;
    }
    // adjoint: sum r S_k of each point over both slices and the KRIG_LOO_REP copies
    // (one warp per point, one copy per lane), the interior orbit sums likewise;
    // the FP64 partial sums enter at FP32 precision (relative 6e-8 each)
    const double* lbar = (const double*)(P.ws + V.lbar_off) + (int64_t)local * (2 * nn);
    const int64_t lrep = (int64_t)V.ncx * V.ncy * (2 * nn);  // stride between the copies
    for (int i = warp; i < n; i += 8) {
        const int dx = i % nx - lx, dy = i / nx - ly;
        const int k0 = (dy + r) * n2r + (dx + r);
        const ff t = ff_two_sum(__double2float_rn(lbar[lane * lrep + k0]),
                                __double2float_rn(lbar[lane * lrep + n2r * n2r + k0]));
        const ff ts = ff_warp_sum(t);
        if (lane == 0) tsum[i] = ts;
    }
    if (local == V.cint && warp == 7) {
        const double* lorb = (const double*)(P.ws + V.lorb_off);
        for (int o = 0; o < (r + 1) * (r + 2) / 2; ++o) {
            const ff t = ff_warp_sum(ff_make(__double2float_rn(lorb[lane * KRIG_NORB + o])));
            if (lane == 0) osum[o] = t;
        }
    }
    __syncthreads();
    // wbar = 2 gL / N * sum r S_k over both slices, N = (n - 2) H W
    const int64_t nvox = (int64_t)(V.n - 2) * V.H * V.W;
    const float nh = (float)nvox;  // N as an exact pair
    const ff nf = {nh, (float)(nvox - (int64_t)nh)};
    const ff coef = ff_div(ff_scale2(ff_from_double(P.grad_loss[v]), 2.0f), nf);
    for (int i = tid; i < n; i += 256) {
        const int dx = i % nx - lx, dy = i / nx - ly;
        ff sum = tsum[i];
        if (local == V.cint) {
            // interior class: the residual kernel kept only orbit sums (both
            // slices); dL/dtheta depends on wbar only through them (the class
            // system and its symmetric right-hand sides are D4-invariant), so
            // each orbit's total is spread evenly over its taps
            const int a = max(abs(dx), abs(dy)), b = min(abs(dx), abs(dy)), o = a * (a + 1) / 2 + b;
            int cnt = 0;
            for (int qy = -r; qy <= r; ++qy)
                for (int qx = -r; qx <= r; ++qx) {
                    const int qa = max(abs(qx), abs(qy)), qb = min(abs(qx), abs(qy));
                    cnt += (qa * (qa + 1) / 2 + qb) == o;
                }
            sum = ff_add(sum, ff_div(osum[o], ff_make((float)cnt)));
        }
        S.B[0][i][2] = ff_mul(coef, sum);
    }
    __syncthreads();
    // third column by the FP32 inverse of the factorised system, then one refinement
    for (int i = tid; i < n; i += 256) {
        const float* ai = &S.M[0][i][ZL - n];
        float x = 0.0f;
        for (int j = 0; j < n; ++j) x = fmaf(ai[j], S.B[0][j][2].hi, x);
        S.M[0][i][2] = x;  // column 2 of the solved rows
    }
    __syncthreads();
    refine(2, 1);
    if (warp == 0) {
        const ff zero = ff_make(0.0f);
        const ff xx = lane < n ? S.X[0][lane][2] : zero;
        const ff aphi = ff_div(ff_warp_sum(xx), svs);
        if (lane < n) abar[lane] = ff_sub(xx, ff_mul(aphi, S.X[0][lane][1]));
    }
    __syncthreads();
    // dL/dtheta_p = sum_i abar_i (dc0_i/dtheta_p - sum_j d(A+B)_ij/dtheta_p w_j), i, j over the points
    // eight threads per point i, each over every eighth j
    ff tp3[3] = {ff_make(0.0f), ff_make(0.0f), ff_make(0.0f)};
    {
        const int i = tid >> 3, q = tid & 7;
        if (i < n) {
            const int dxi = S.dx[i], dyi = S.dy[i];
            const int i0 = abs(dyi) * nr + abs(dxi);
            ff acc[3] = {ff_make(0.0f), ff_make(0.0f), ff_make(0.0f)};
            if (q == 0) {
#pragma unroll
                for (int p = 0; p < 3; ++p) acc[p] = d0[p][i0];
            }
            for (int j = q; j < n; j += 8) {
                const int ic = abs(dyi - S.dy[j]) * n2r + abs(dxi - S.dx[j]);
#pragma unroll
                for (int p = 0; p < 3; ++p) acc[p] = ff_sub(acc[p], ff_mul(ff_add(dC[p][ic], dC[p][nn + ic]), wgt[j]));
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) tp3[p] = ff_mul(abar[i], acc[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) tp3[p] = ff_warp_sum(tp3[p]);
    if (lane == 0) {
#pragma unroll
        for (int p = 0; p < 3; ++p) red[warp][p] = tp3[p];
    }
    __syncthreads();
    if (tid < 3) {
        ff s = red[0][tid];
        for (int w = 1; w < 8; ++w) s = ff_add(s, red[w][tid]);
        atomicAdd(P.grad_params + 3 * v + tid, ff_to_double(s));
    }
}

// ---------------------------------------------------------------------------
// Residual kernel: one block per (volume, target slice j, 64 x 16 tile).
// mode 0: loss (and optional prediction).  mode 1: residual buffer and the
// interior class's sums r * (orbit sum) for dL/dw (the border classes' tap sums
// are formed from the stored residuals by loo_border_block).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float loo_load(const void* in, int dtype, float scale, size_t idx)
{
    if (dtype == KRIG_F32) return ((const float*)in)[idx];
    if (dtype == KRIG_U16) return __fmul_rn((float)((const uint16_t*)in)[idx], scale);
    return (float)((const double*)in)[idx];
}

// Four consecutive elements of a slice as float, starting at element idx
// (idx and the row width multiples of 4, all four inside the row).
__device__ __forceinline__ void loo_load4(const void* in, int dtype, float scale, size_t idx, float o[4])
{
    if (dtype == KRIG_F32) {
        const float4 a = *(const float4*)((const float*)in + idx);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    } else if (dtype == KRIG_U16) {
        const uint2 a = *(const uint2*)((const uint16_t*)in + idx);
        o[0] = __fmul_rn((float)(a.x & 0xffffu), scale);
        o[1] = __fmul_rn((float)(a.x >> 16), scale);
        o[2] = __fmul_rn((float)(a.y & 0xffffu), scale);
        o[3] = __fmul_rn((float)(a.y >> 16), scale);
    } else {
        const double2 a = *(const double2*)((const double*)in + idx), b = *(const double2*)((const double*)in + idx + 2);
        o[0] = (float)a.x; o[1] = (float)a.y; o[2] = (float)b.x; o[3] = (float)b.y;
    }
}

// Tile staging in two phases: loo_fetch issues every global load of the
// thread into registers, loo_commit converts and stores them to shared memory.
// A block then waits for one memory latency per tile set instead of one per
// loop step.  The tile is ROWS rows x 4G columns from (ytop, xleft) of slice
// `plane_off`, zeros outside the slice (xleft, the row width and the slice
// width multiples of 4 on the vector path).
template <int ROWS, int G>
struct LooStage {
    static constexpr int NIT = (ROWS * G + 255) / 256;
    uint4 raw[NIT];
    unsigned conv;  // bit it: raw[it] holds four u16 values still to be scaled
};

template <int ROWS, int G>
__device__ __forceinline__ void loo_fetch(const void* in, int dtype, float scale, size_t plane_off, int H, int W,
                                          int ytop, int xleft, LooStage<ROWS, G>& st, int tid)
{
    const bool vec = (W & 3) == 0 && dtype != KRIG_F64;
    st.conv = 0u;
#pragma unroll
    for (int it = 0; it < LooStage<ROWS, G>::NIT; ++it) {
        const int e = tid + it * 256;
        st.raw[it] = make_uint4(0u, 0u, 0u, 0u);
        if (e >= ROWS * G) continue;
        const int yy = ytop + e / G, xx = xleft + (e % G) * 4;
        if (yy < 0 || yy >= H) continue;
        const size_t row = plane_off + (size_t)yy * W;
        if (vec && xx >= 0 && xx + 3 < W) {
            if (dtype == KRIG_F32) {
                st.raw[it] = *(const uint4*)((const float*)in + row + xx);
            } else {
                const uint2 a = *(const uint2*)((const uint16_t*)in + row + xx);
                st.raw[it].x = a.x;
                st.raw[it].y = a.y;
                st.conv |= 1u << it;
            }
        } else {
            float f[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (xx + q >= 0 && xx + q < W) f[q] = loo_load(in, dtype, scale, row + xx + q);
            st.raw[it] = make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]),
                                    __float_as_uint(f[3]));
        }
    }
}

template <int ROWS, int G>
__device__ __forceinline__ void loo_commit(const LooStage<ROWS, G>& st, float scale, float* dst, int tid)
{
    static_assert(4 * G <= LOO_SP, "tile row wider than the shared-memory stride");
#pragma unroll
    for (int it = 0; it < LooStage<ROWS, G>::NIT; ++it) {
        const int e = tid + it * 256;
        if (e >= ROWS * G) continue;
        const uint4 a = st.raw[it];
        float4 f;
        if ((st.conv >> it) & 1u) {
            f.x = __fmul_rn((float)(a.x & 0xffffu), scale);
            f.y = __fmul_rn((float)(a.x >> 16), scale);
            f.z = __fmul_rn((float)(a.y & 0xffffu), scale);
            f.w = __fmul_rn((float)(a.y >> 16), scale);
        } else {
            f = make_float4(__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z), __uint_as_float(a.w));
        }
        *(float4*)(dst + (e / G) * LOO_SP + (e % G) * 4) = f;
    }
}

// The LOO weight table and the orbit weights after it (nw floats, a multiple
// of four, at most 2048) into shared memory, loads first.
__device__ __forceinline__ void loo_copy_weights(const float* lwg, int nw, float* dst, int tid)
{
    float4 a[2];
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int e = tid + it * 256;
        a[it] = e * 4 < nw ? ((const float4*)lwg)[e] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int e = tid + it * 256;
        if (e * 4 < nw) ((float4*)dst)[e] = a[it];
    }
}

// D4 orbit sums of a + b (two tiles with the residual-kernel layout) around
// the four pixels of a thread: the LOO interior class is D4-symmetric and has
// the same weights in both slices, so its stencil is sum_o w_o * orbit sum.
template <int R> struct LooNO { static constexpr int N = R == 0 ? 1 : (R == 1 ? 3 : 6); };

template <int R>
__device__ __forceinline__ void loo_orbits(const float* a, const float* b, int lrow, int lcol,
                                           float (&o)[4][LooNO<R>::N])
{
    static_assert(LOO_PAD == 4 && R <= 4, "window columns lcol - 4 .. lcol + 7 cover the taps");
    constexpr int NC = 4 + 2 * R;
    float F[2 * R + 1][NC];
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
        // the 16-byte-aligned columns lcol - 4 .. lcol + 7 of both rows, three vector loads each
        const int base = (lrow + R + dy) * LOO_SP + lcol;
        float wa[12], wb[12];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (R == 0 && q != 1) continue;
            const float4 u = *(const float4*)(a + base + 4 * q), t = *(const float4*)(b + base + 4 * q);
            wa[4 * q] = u.x; wa[4 * q + 1] = u.y; wa[4 * q + 2] = u.z; wa[4 * q + 3] = u.w;
            wb[4 * q] = t.x; wb[4 * q + 1] = t.y; wb[4 * q + 2] = t.z; wb[4 * q + 3] = t.w;
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) F[dy + R][k] = wa[4 - R + k] + wb[4 - R + k];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int m = R + p;
        o[p][0] = F[R][m];
        if (R >= 1) {
            o[p][1] = (F[R][m - 1] + F[R][m + 1]) + (F[R - 1][m] + F[R + 1][m]);
            o[p][2] = (F[R - 1][m - 1] + F[R - 1][m + 1]) + (F[R + 1][m - 1] + F[R + 1][m + 1]);
        }
        if (R >= 2) {
            o[p][3] = (F[R][m - 2] + F[R][m + 2]) + (F[R - 2][m] + F[R + 2][m]);
            o[p][4] = ((F[R - 1][m - 2] + F[R - 1][m + 2]) + (F[R + 1][m - 2] + F[R + 1][m + 2])) +
                      ((F[R - 2][m - 1] + F[R - 2][m + 1]) + (F[R + 2][m - 1] + F[R + 2][m + 1]));
            o[p][5] = (F[R - 2][m - 2] + F[R - 2][m + 2]) + (F[R + 2][m - 2] + F[R + 2][m + 2]);
        }
    }
}

// One chain item: targets j in [ja, jb) of the tile at (x0, y0).  Four slice
// buffers (tile plus halo) rotate in shared memory: target j reads j - 1, j and
// j + 1; slice j + 2, loaded into registers during the previous step, is
// stored after it, while the loads of slice j + 3 are in flight, so each slice
// of the chain is read once and a load has two steps to arrive.  The
// loss and (mode 1) the interior orbit sums stay in registers over the chain
// and are reduced once, into copy rep of the accumulators.
template <int R>
__device__ void loo_residual_chain(const KrigLaunch& P, int v, int ja, int jb, int x0, int y0, int mode, int rep,
                                   float* sm)
{
    constexpr int N2R = 2 * R + 1, NTAP = 2 * N2R * N2R;
    constexpr int ROWS = LOO_TY + 2 * R;
    constexpr int BUF = ROWS * LOO_SP;
    const KrigVol& V = P.vol[v];
    const int H = V.H, W = V.W;
    const size_t plane = (size_t)H * W;
    float* wsm = sm + 4 * BUF;                        // [ncls][NTAP] LOO weights, orbit weights
    float* sgo = wsm + loo_wo_off(25 * NTAP) + 8;     // interior sum r * orbit sum (mode 1)
    double* sl = (double*)(sgo + 8);                  // loss partials of the warps (8)
    constexpr int NO = LooNO<R>::N;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncls = V.ncx * V.ncy;
    const float* wo = wsm + loo_wo_off(ncls * NTAP);  // interior weight per orbit
    const float* lw = wsm;
    const auto buf = [&](int s) { return sm + (s & 3) * BUF; };
    const auto fetch = [&](int s, LooStage<ROWS, LOO_RP / 4>& st) {
        loo_fetch(P.in[v], V.dtype, V.scale, (size_t)s * plane, H, W, y0 - R, x0 - LOO_PAD, st, tid);
    };
    {
        LooStage<ROWS, LOO_RP / 4> a, b, c;
        fetch(ja - 1, a);
        fetch(ja, b);
        fetch(ja + 1, c);
        loo_copy_weights((const float*)(P.ws + V.lw_off), loo_wo_off(ncls * NTAP) + 8, wsm, tid);
        loo_commit(a, V.scale, buf(ja - 1), tid);
        loo_commit(b, V.scale, buf(ja), tid);
        loo_commit(c, V.scale, buf(ja + 1), tid);
        if (tid < 8) sgo[tid] = 0.f;
    }
    __syncthreads();
    const int lrow = (warp >> 2) * 8 + (lane >> 2);
    const int lcol = (warp & 3) * 16 + (lane & 3) * 4;
    const int y = y0 + lrow;
    float gio[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) gio[o] = 0.f;
    double loss = 0.0;
    const bool row_in = V.cint >= 0 && y >= R && y <= H - 1 - R;
    const bool all_in = row_in && x0 + lcol >= R && x0 + lcol + 3 <= W - 1 - R;
    float* dst = mode == 0 ? P.pred[v] : (float*)(P.ws + V.res_off);
    LooStage<ROWS, LOO_RP / 4> nx, nx2;  // slices j + 2 (loaded) and j + 3 (in flight)
    if (ja + 2 <= jb) fetch(ja + 2, nx);
    for (int j = ja; j < jb; ++j) {
        const bool more = j + 2 <= jb;   // slice j + 2 brackets target j + 1
        const bool more2 = j + 3 <= jb;
        if (more2) fetch(j + 3, nx2);
        const float* lo = buf(j - 1);
        const float* hi = buf(j + 1);
        const float* ce = buf(j) + R * LOO_SP + LOO_PAD;  // the target slice, tile rows and columns
        float loss4 = 0.f;  // the thread's (at most four) squared residuals, FP32
        float outv[4] = {0.f, 0.f, 0.f, 0.f};
        if (y < H) {
            float cev[4];
            {
                const float4 c4 = *(const float4*)(ce + lrow * LOO_SP + lcol);
                cev[0] = c4.x; cev[1] = c4.y; cev[2] = c4.z; cev[3] = c4.w;
            }
            // interior pixels: orbit sums of the two slices, one FMA per orbit
            float orb[4][NO];
            if (row_in) loo_orbits<R>(lo, hi, lrow, lcol, orb);
            // residual, loss term and output of pixel p; interior pixels also feed the
            // orbit sums of dL/dw (border classes: loo_border_block, from the stored residuals)
            const auto finish = [&](int p, float pred, bool inner) {
                const float res = pred - cev[p];
                loss4 = fmaf(res, res, loss4);
                outv[p] = mode == 0 ? pred : res;
                if (mode == 1 && inner) {
#pragma unroll
                    for (int o = 0; o < NO; ++o) gio[o] = fmaf(res, orb[p][o], gio[o]);
                }
            };
            if (all_in) {
                // all four pixels in the interior class
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float pred = 0.f;
#pragma unroll
                    for (int o = 0; o < NO; ++o) pred = fmaf(wo[o], orb[p][o], pred);
                    finish(p, pred, true);
                }
            } else {
                const int cy = V.ymap[krig_slot(y, H, R)];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int x = x0 + lcol + p;
                    if (x >= W) break;
                    const int c = cy * V.ncx + V.xmap[krig_slot(x, W, R)];
                    const bool inner = row_in && c == V.cint;
                    float pred = 0.f;
                    if (inner) {
#pragma unroll
                        for (int o = 0; o < NO; ++o) pred = fmaf(wo[o], orb[p][o], pred);
                    } else {
                        const float* wr = lw + (int64_t)c * NTAP;
#pragma unroll
                        for (int s = 0; s < 2; ++s)
#pragma unroll
                            for (int dy = -R; dy <= R; ++dy)
#pragma unroll
                                for (int dx = -R; dx <= R; ++dx) {
                                    const int k = (s * N2R + (dy + R)) * N2R + (dx + R);
                                    pred = fmaf(wr[k],
                                                (s == 0 ? lo : hi)[(lrow + R + dy) * LOO_SP + LOO_PAD + lcol + p + dx],
                                                pred);
                                }
                    }
                    finish(p, pred, inner);
                }
            }
            // predictions (mode 0, when asked for) or residuals (mode 1): one vector store
            // when the four pixels are in the slice and the row is 16-byte aligned
            if (dst) {
                const size_t oidx = (size_t)(j - 1) * plane + (size_t)y * W + x0 + lcol;
                if ((W & 3) == 0 && x0 + lcol + 3 < W) {
                    *(float4*)(dst + oidx) = make_float4(outv[0], outv[1], outv[2], outv[3]);
                } else {
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        if (x0 + lcol + p < W) dst[oidx + p] = outv[p];
                }
            }
        }
        loss += (double)loss4;
        if (more) loo_commit(nx, V.scale, buf(j + 2), tid);  // buffer of slice j - 2: read last by step j - 1
        nx = nx2;
        __syncthreads();
    }
    // loss: warp (FP64) -> block -> volume accumulator
    for (int o = 16; o; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) sl[warp] = loss;
    if (mode == 1 && V.cint >= 0) {
#pragma unroll
        for (int o = 0; o < NO; ++o) {
            float t = gio[o];
            for (int k = 16; k; k >>= 1) t += __shfl_xor_sync(0xffffffffu, t, k);
            if (lane == 0) atomicAdd(&sgo[o], t);
        }
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sl[w];
        atomicAdd((double*)(P.ws + V.lacc_off) + rep, s);
    }
    if (mode == 1 && V.cint >= 0 && tid < NO && sgo[tid] != 0.f)
        atomicAdd((double*)(P.ws + V.lorb_off) + rep * KRIG_NORB + tid, (double)sgo[tid]);
    __syncthreads();  // the next item overwrites the buffers, the weights and sgo
}

// ---------------------------------------------------------------------------
// Tap sums sum_p r(p) S(p + d_k) of the border classes (backward pass): one
// block per (volume, class, target slice j, bracketing slice s).  A class's
// pixels form a rectangle (a row or column segment at the border, or one
// corner pixel); each thread takes pixels of it and keeps one sum per tap of
// slice s, then the block reduces them and adds them into one of the
// KRIG_LOO_REP copies.  Runs as the first blocks of the gradient launch.
// ---------------------------------------------------------------------------
__host__ __device__ inline int64_t loo_border_blocks(const KrigVol& V) { return 2LL * V.ncx * V.ncy * (V.n - 2); }

template <int R>
__device__ void loo_border_block(const KrigLaunch& P, int64_t b, float* sm)
{
    constexpr int N2R = 2 * R + 1, NT = N2R * N2R;  // taps of one slice
    int64_t acc0 = 0;
    int v = -1;
    for (int u = 0; u < P.n_vols; ++u) {
        const int64_t cnt = loo_border_blocks(P.vol[u]);
        if (b < acc0 + cnt) {
            v = u;
            break;
        }
        acc0 += cnt;
    }
    if (v < 0) return;
    const KrigVol& V = P.vol[v];
    if (V.r != R) return;
    const int ncls = V.ncx * V.ncy;
    const int local = (int)(b - acc0), cls = local % ncls, s = (local / ncls) & 1, j = 1 + local / (2 * ncls);
    if (cls == V.cint) return;  // interior: orbit sums in the residual kernel
    const int cy = cls / V.ncx, cx = cls % V.ncx;
    const int H = V.H, W = V.W;
    const int ly = V.yext[cy][0], ry = V.yext[cy][1], lx = V.xext[cx][0], rx = V.xext[cx][1];
    // the class's rows and columns: a truncated side fixes the coordinate
    const int ya = ly < R ? ly : (ry < R ? H - 1 - ry : R), yb = ly < R ? ly : (ry < R ? H - 1 - ry : H - 1 - R);
    const int xa = lx < R ? lx : (rx < R ? W - 1 - rx : R), xb = lx < R ? lx : (rx < R ? W - 1 - rx : W - 1 - R);
    const int nxr = xb - xa + 1, npx = (yb - ya + 1) * nxr;
    const size_t plane = (size_t)H * W;
    const float* res = (const float*)(P.ws + V.res_off) + (size_t)(j - 1) * plane;
    const size_t sl = (size_t)(j - 1 + 2 * s) * plane;  // slice j - 1 (s = 0) or j + 1 (s = 1)
    float acc[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) acc[k] = 0.f;
    for (int q = threadIdx.x; q < npx; q += 256) {
        const int y = ya + q / nxr, x = xa + q % nxr;
        const float rr = res[(size_t)y * W + x];
#pragma unroll
        for (int dy = -R; dy <= R; ++dy)
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                if (dy < -ly || dy > ry || dx < -lx || dx > rx) continue;  // truncated tap
                const int k = (dy + R) * N2R + (dx + R);
                acc[k] = fmaf(rr, loo_load(P.in[v], V.dtype, V.scale, sl + (size_t)(y + dy) * W + (x + dx)), acc[k]);
            }
    }
    float* red = sm;  // [8][NT]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        float t = acc[k];
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[warp * NT + k] = t;
    }
    __syncthreads();
    if (threadIdx.x < NT) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += red[w * NT + threadIdx.x];
        if (t != 0.f) {
            const int rep = (int)(b % KRIG_LOO_REP);
            double* lbar = (double*)(P.ws + V.lbar_off) + (int64_t)rep * ncls * 2 * NT;
            atomicAdd(lbar + (int64_t)cls * 2 * NT + s * NT + threadIdx.x, (double)t);
        }
    }
}

// One instance per half-width r (the tap arrays set the register budget);
// blocks of volumes with another r leave at once.
template <int R>
__global__ void __launch_bounds__(256, 2) k_loo_residual(const __grid_constant__ KrigLaunch P, int mode)
{
    extern __shared__ __align__(16) float lsm[];
    asm volatile("griddepcontrol.launch_dependents;");
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the class weights of this pass
    // a grid of resident blocks walks the chain items (it = blockIdx.x mod gridDim.x)
    for (int64_t it = blockIdx.x; it < P.n_loo_items; it += gridDim.x) {
        int v = 0;
        for (int u = 1; u < P.n_vols; ++u)
            if (P.vol[u].loo_item_begin <= it) v = u;
        const KrigVol& V = P.vol[v];
        if (V.r != R) continue;
        const int64_t local = it - V.loo_item_begin;
        const int tiles = V.tiles_x * V.tiles_y;
        const int chunk = (int)(local / tiles);
        const int tile = (int)(local % tiles);
        const int x0 = (tile % V.tiles_x) * LOO_TX, y0 = (tile / V.tiles_x) * LOO_TY;
        const int ja = 1 + chunk * KRIG_LOO_CHAIN, jb = min(ja + KRIG_LOO_CHAIN, V.n - 1);
        loo_residual_chain<R>(P, v, ja, jb, x0, y0, mode, (int)(it % KRIG_LOO_REP), lsm);
    }
    if (mode != 0) return;
    // forward: the last block of the launch turns the loss sums of the volumes
    // with this r into their losses (thread 0 of every block made its loss
    // atomic before its fence and ticket); the ticket counter resets itself
    __shared__ unsigned last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned* done = (unsigned*)(P.ws + KRIG_CTRL_LOO_DONE);
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int u = threadIdx.x; u < P.n_vols; u += blockDim.x) {
        const KrigVol& U = P.vol[u];
        if (U.r != R) continue;
        const double* acc = (const double*)(P.ws + U.lacc_off);
        double sum = 0.0;
        for (int c = 0; c < KRIG_LOO_REP; ++c) sum += __ldcg(acc + c);
        P.loss[u] = sum / ((double)(U.n - 2) * U.H * U.W);
    }
    if (threadIdx.x == 0) *(unsigned*)(P.ws + KRIG_CTRL_LOO_DONE) = 0u;
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
    float* rdn = sm + ROWS * LOO_SP;   // r_{m-1}: predictions for which S_m is the upper slice
    float* wsm = rdn + ROWS * LOO_SP;  // [ncls][NTAP] LOO weights, orbit weights
    constexpr int NO = LooNO<R>::N;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float* wo = wsm + loo_wo_off(V.ncx * V.ncy * NTAP);  // interior weight per orbit
    const bool has_up = m + 1 <= n - 2, has_dn = m - 1 >= 1;
    const int lrow = (warp >> 2) * 8 + (lane >> 2);
    const int lcol = (warp & 3) * 16 + (lane & 3) * 4;
    const int y = y0 + lrow;
    float* gs = P.grad_slices[v];
    float rc[4], gprev[4];
    {
        // r_{m+1} sits at residual index m, r_{m-1} at m-2 (zero tiles past the ends:
        // the fetch of a row outside 0..H-1 loads nothing)
        LooStage<ROWS, LOO_RP / 4> a, b;
        loo_fetch(res, KRIG_F32, 1.0f, (size_t)(has_up ? m : 0) * plane, has_up ? H : 0, W, y0 - R, x0 - LOO_PAD, a,
                  tid);
        loo_fetch(res, KRIG_F32, 1.0f, (size_t)(has_dn ? m - 2 : 0) * plane, has_dn ? H : 0, W, y0 - R,
                  x0 - LOO_PAD, b, tid);
        loo_copy_weights((const float*)(P.ws + V.lw_off), loo_wo_off(V.ncx * V.ncy * NTAP) + 8, wsm, tid);
        // the thread's own residuals r_m and (accumulating) the previous gradient, loaded
        // with the tiles
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int x = x0 + lcol + p;
            rc[p] = 0.f;
            gprev[p] = 0.f;
            if (y < H && x < W) {
                if (m >= 1 && m <= n - 2) rc[p] = res[(size_t)(m - 1) * plane + (size_t)y * W + x];
                if (P.accumulate) gprev[p] = gs[(size_t)m * plane + (size_t)y * W + x];
            }
        }
        loo_commit(a, 1.0f, rup, tid);
        loo_commit(b, 1.0f, rdn, tid);
    }
    __syncthreads();
    if (y >= H) return;
    const float* lw = wsm;
    const double coef = 2.0 * P.grad_loss[v] / ((double)(n - 2) * H * W);
    const float fcoef = (float)coef;
    // pixels whose whole window lies in the interior class (2r from the
    // border): sum_o w_o * orbit sum of (r_{m+1} + r_{m-1})
    const bool row_in = V.cint >= 0 && y >= 2 * R && y <= H - 1 - 2 * R;
    float orb[4][NO];
    if (row_in) loo_orbits<R>(rup, rdn, lrow, lcol, orb);
    float outv[4] = {0.f, 0.f, 0.f, 0.f};
    const bool all_in = row_in && x0 + lcol >= 2 * R && x0 + lcol + 3 <= W - 1 - 2 * R;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int x = x0 + lcol + p;
        if (!all_in && x >= W) break;
        float acc = 0.f;
        if (all_in || (row_in && x >= 2 * R && x <= W - 1 - 2 * R)) {
#pragma unroll
            for (int o = 0; o < NO; ++o) acc = fmaf(wo[o], orb[p][o], acc);
        } else {
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
                const int off = (lrow + R - dy) * LOO_SP + LOO_PAD + lcol + p - dx;
                acc = fmaf(wr[(0 * N2R + (dy + R)) * N2R + (dx + R)], rup[off], acc);  // S_m lower of m+1
                acc = fmaf(wr[(1 * N2R + (dy + R)) * N2R + (dx + R)], rdn[off], acc);  // S_m upper of m-1
            }
        }
        }
        // FP32: the per-pixel terms need no FP64 (FP64 issues at 1/64 rate)
        const float gval = (acc - rc[p]) * fcoef;
        outv[p] = P.accumulate ? gprev[p] + gval : gval;
    }
    const size_t oidx = (size_t)m * plane + (size_t)y * W + x0 + lcol;
    if ((W & 3) == 0 && x0 + lcol + 3 < W) {
        *(float4*)(gs + oidx) = make_float4(outv[0], outv[1], outv[2], outv[3]);
    } else {
#pragma unroll
        for (int p = 0; p < 4; ++p)
            if (x0 + lcol + p < W) gs[oidx + p] = outv[p];
    }
}

// Gradient launch: blocks [0, nborder) form the border-class tap sums (dL/dw,
// for dL/dtheta), the rest the adjoint w.r.t. the slices; both read only the
// residuals, so they share one launch.
template <int R>
__global__ void __launch_bounds__(256, R == 2 ? 3 : 4) k_loo_grad(const __grid_constant__ KrigLaunch P, int64_t nborder)
{
    extern __shared__ __align__(16) float lsm[];
    asm volatile("griddepcontrol.launch_dependents;");
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the residuals of this pass
    if ((int64_t)blockIdx.x < nborder) {
        loo_border_block<R>(P, blockIdx.x, lsm);
        return;
    }
    const int64_t it = blockIdx.x - nborder;
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
    if (V.r == R) loo_adjoint_tile<R>(P, v, m, x0, y0, lsm);
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
        const size_t wcap = (size_t)loo_wo_off(25 * ntap) + 8;  // weights + orbit weights
        size_t b = adjoint ? ((size_t)2 * rows * LOO_SP + wcap) * 4 : ((size_t)4 * rows * LOO_SP + wcap + 8) * 4 + 8 * 8;
        if (b > m) m = b;
    }
    return m;
}

// Every LOO kernel waits for its predecessor on the stream (griddepcontrol.wait)
// before it touches the pass's data, so each kernel after the first of a pass
// is launched early (programmatic dependent launch): its blocks are scheduled
// while the previous grid drains.  The first kernel of a pass is an ordinary
// launch: it starts after whatever the caller queued before it (which may
// write the variogram parameters) has completed, so the kernels chained
// behind it may read those parameters before their own wait.
template <typename... KArgs, typename... Args>
static cudaError_t loo_launch(bool early, void (*kernel)(KArgs...), unsigned grid, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = early ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

int krig_launch_loo(const KrigLaunch& L, int backward, int want_grad_slices, int want_grad_params, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    // the class launch also zeroes the accumulators of the pass
    if ((e = loo_launch(false, k_loo_class, (unsigned)L.n_loo_classes, 0, st, L, backward ? 2 : 0)) != cudaSuccess) return (int)e;
    bool has_r[KRIG_RMAX + 1] = {};
    for (int v = 0; v < L.n_vols; ++v) has_r[L.vol[v].r] = true;
    const size_t s1 = loo_smem(L, 0);
    // resident blocks of the residual kernel: two per SM (its launch bounds)
    const unsigned g1 = (unsigned)std::min<int64_t>(L.n_loo_items, (int64_t)2 * krig_device_sm_count());
    for (int r = 0; r <= KRIG_RMAX; ++r) {
        if (!has_r[r]) continue;
        const int mode = backward ? 1 : 0;
        if (r == 0) e = loo_launch(true, k_loo_residual<0>, g1, s1, st, L, mode);
        else if (r == 1) e = loo_launch(true, k_loo_residual<1>, g1, s1, st, L, mode);
        else e = loo_launch(true, k_loo_residual<2>, g1, s1, st, L, mode);
        if (e != cudaSuccess) return (int)e;
    }
    if (!backward) return 0;
    int64_t nb = 0;
    if (want_grad_params)
        for (int v = 0; v < L.n_vols; ++v) nb += loo_border_blocks(L.vol[v]);
    const int64_t na = want_grad_slices ? L.n_loo_adj : 0;
    if (nb + na > 0) {
        const size_t s2 = loo_smem(L, 1);
        for (int r = 0; r <= KRIG_RMAX; ++r) {
            if (!has_r[r]) continue;
            if (r == 0) e = loo_launch(true, k_loo_grad<0>, (unsigned)(nb + na), s2, st, L, nb);
            else if (r == 1) e = loo_launch(true, k_loo_grad<1>, (unsigned)(nb + na), s2, st, L, nb);
            else e = loo_launch(true, k_loo_grad<2>, (unsigned)(nb + na), s2, st, L, nb);
            if (e != cudaSuccess) return (int)e;
        }
    }
    if (want_grad_params) {
        if ((e = loo_launch(true, k_loo_class, (unsigned)L.n_loo_classes, 0, st, L, 1)) != cudaSuccess) return (int)e;
    }
    return 0;
}
