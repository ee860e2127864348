// krig_ds.cu -- the deduplicated-stencil (DS) form of the kriging path.
//
// A missing voxel's kriging system depends only on its geometry: its offset t
// inside the gap and how its (2r+1)^2 window is truncated at the in-plane
// border (Sec. 4.1.2: the system is built from distances between the target
// and its neighbouring known voxels; Appendix A: the weights solve the
// extended covariance system).  So the weights are solved once per
// truncation class (k_ds_solve, one block per (y-class, x-class), all t at
// once) and applied to every voxel as a stencil over the two bracketing known
// slices (k_ds_apply).  k_ds_apply walks the work items of Algorithm 1: each
// item is one in-plane tile of one Z sub-block; it stages the sub-block's
// known slices through shared memory one at a time, so every known slice of
// the block is read from memory once, and writes the block's output slices
// (including the bit-exact copy of its known slices, Algorithm 1 step 3)
// straight to their final offsets (the merge of Sec. 4.2).
#include <cuda_runtime.h>
#include <stdint.h>

#include "krig_device.cuh"

// ---------------------------------------------------------------------------
// Class solve: one block of 256 threads per xy-class.
// ---------------------------------------------------------------------------

template <typename TF>
__global__ void __launch_bounds__(256) k_ds_solve(const __grid_constant__ KrigLaunch P)
{
    __shared__ SolveSmem<TF, KRIG_KMAX, 8> S;
    __shared__ double gC[2 * (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1)];
    __shared__ double g0[(KRIG_GMAX - 1) * 2 * (KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    __shared__ double phi[8], vout[8];

    const int tid = threadIdx.x;
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

    const int lx = V.xext[cx][0], rx = V.xext[cx][1], ly = V.yext[cy][0], ry = V.yext[cy][1];
    const int nx = lx + rx + 1, ny = ly + ry + 1;
    const int K = 2 * nx * ny;
    const int NC = V.g;  // g-1 targets + ones
    for (int i = tid; i < K; i += 256) {
        Tap tp;
        tp.s = (int8_t)(i / (nx * ny));
        tp.dy = (int8_t)((i / nx) % ny - ly);
        tp.dx = (int8_t)(i % nx - lx);
        tp.pad = 0;
        S.tap[i] = tp;
    }
    __syncthreads();
    for (int e = tid; e < K * NC; e += 256) {
        int i = e / NC, c = e % NC;
        Tap tp = S.tap[i];
        S.Bd[i * 8 + c] = c < NC - 1 ? g0[d.i0(c + 1, tp.s, abs(tp.dy), abs(tp.dx))] : 1.0;
    }
    __syncthreads();
    const bool ok = team_ok_solve<TF, KRIG_KMAX, 8, 256>(S, d, gC, K, NC, tid);
    if (!ok && tid == 0) krig_set_status(P.status, KRIG_DEV_SINGULAR);
    if (tid < 32 && ok) {
        // phi_c = (1'u_c - 1) / (1'v); var_c = C(0) - w_c'c0_c - phi_c
        double sv = 0.0;
        for (int i = tid; i < K; i += 32) sv += S.Xd[i * 8 + NC - 1];
        for (int o = 16; o; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
        for (int c = 0; c < NC - 1; ++c) {
            double su = 0.0, wc = 0.0;
            for (int i = tid; i < K; i += 32) su += S.Xd[i * 8 + c];
            for (int o = 16; o; o >>= 1) su += __shfl_xor_sync(0xffffffffu, su, o);
            double ph = (su - 1.0) / sv;
            for (int i = tid; i < K; i += 32) wc += (S.Xd[i * 8 + c] - ph * S.Xd[i * 8 + NC - 1]) * S.Bd[i * 8 + c];
            for (int o = 16; o; o >>= 1) wc += __shfl_xor_sync(0xffffffffu, wc, o);
            if (tid == 0) {
                phi[c] = ph;
                vout[c] = gC[0] - wc - ph;
            }
        }
    }
    __syncthreads();
    // Weight table row of this class: [s][dy+r][dx+r][t slot], zeros on
    // truncated taps and unused t slots.  u16 input: weights carry the scale.
    const int n2r = 2 * r + 1;
    const int ntap = 2 * n2r * n2r;
    const double scale = V.dtype == KRIG_U16 ? (double)V.scale : 1.0;
    const int64_t row = ((int64_t)cy * V.ncx + cx) * ntap * KRIG_TSLOTS;
    for (int e = tid; e < ntap * KRIG_TSLOTS; e += 256) {
        int c = e % KRIG_TSLOTS, f = e / KRIG_TSLOTS;
        int dx = f % n2r - r, dy = (f / n2r) % n2r - r, s = f / (n2r * n2r);
        double w = 0.0;
        if (c < NC - 1 && dx >= -lx && dx <= rx && dy >= -ly && dy <= ry) {
            int i = (s * ny + (dy + ly)) * nx + (dx + lx);
            w = ok ? (S.Xd[i * 8 + c] - phi[c] * S.Xd[i * 8 + NC - 1]) * scale : __longlong_as_double(0x7ff8000000000000LL);
        }
        if (V.dtype == KRIG_F64) ((double*)(P.ws + V.wtab_off))[row + e] = w;
        else ((float*)(P.ws + V.wtab_off))[row + e] = (float)w;
    }
    if (tid < KRIG_TSLOTS) {
        float* vt = (float*)(P.ws + V.vtab_off) + ((int64_t)cy * V.ncx + cx) * KRIG_TSLOTS;
        vt[tid] = (tid < NC - 1) ? (ok ? (float)vout[tid] : __int_as_float(0x7fc00000)) : 0.0f;
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

// ---------------------------------------------------------------------------
// Stencil apply: persistent blocks over (volume, sub-block, tile) items.
// ---------------------------------------------------------------------------

template <typename TI> struct DsTypes;
template <> struct DsTypes<double> { typedef double TC; typedef double TO; static constexpr int PAD = 4; };
template <> struct DsTypes<float> { typedef float TC; typedef float TO; static constexpr int PAD = 4; };
template <> struct DsTypes<uint16_t> { typedef float TC; typedef float TO; static constexpr int PAD = 8; };

// four consecutive shared-memory elements, widened to the compute type
__device__ __forceinline__ void ld4(const double* p, double o[4])
{
    double2 a = *(const double2*)p, b = *(const double2*)(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4(const float* p, float o[4])
{
    float4 a = *(const float4*)p;
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void ld4(const uint16_t* p, float o[4])
{
    uint2 a = *(const uint2*)p;
    o[0] = (float)(a.x & 0xffffu); o[1] = (float)(a.x >> 16); o[2] = (float)(a.y & 0xffffu); o[3] = (float)(a.y >> 16);
}

// eight t-slot weights of one tap
__device__ __forceinline__ void ldw(const float* p, float w[8])
{
    float4 a = __ldg((const float4*)p), b = __ldg((const float4*)(p + 4));
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}
__device__ __forceinline__ void ldw(const double* p, double w[8])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double2 a = __ldg((const double2*)(p + 2 * q));
        w[2 * q] = a.x; w[2 * q + 1] = a.y;
    }
}

// exact value of a stored input element (u16: float32(u) * scale)
__device__ __forceinline__ double cvt_out(double x, float) { return x; }
__device__ __forceinline__ float cvt_out(float x, float) { return x; }
__device__ __forceinline__ float cvt_out(uint16_t u, float scale) { return __fmul_rn((float)u, scale); }

template <typename T>
__device__ __forceinline__ void st4(T* p, const T v[4], bool vec_ok, int nvalid)
{
    if (vec_ok) {
        if (sizeof(T) == 4) {
            __stcs((float4*)p, make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]));
        } else {
            __stcs((double2*)p, make_double2((double)v[0], (double)v[1]));
            __stcs((double2*)p + 1, make_double2((double)v[2], (double)v[3]));
        }
    } else {
        for (int p_ = 0; p_ < 4; ++p_)
            if (p_ < nvalid) p[p_] = v[p_];
    }
}

// Stage the tile + halo of one known slice into shared memory; zeros outside
// the volume (they meet zero weights of truncated taps).
template <typename TI, int R>
__device__ __forceinline__ void ds_fill(TI* slot, const TI* src, int x0, int y0, int H, int W, bool vec_rows)
{
    constexpr int PAD = DsTypes<TI>::PAD;
    constexpr int RP = KRIG_TX + 2 * PAD;
    constexpr int ROWS = KRIG_TY + 2 * R;
    constexpr int VEC = 16 / sizeof(TI);
    if (vec_rows) {
        // 16-byte chunks: x0 - PAD and W are multiples of VEC, so a chunk is
        // wholly inside or wholly outside [0, W).
        constexpr int CPR = RP / VEC;
        for (int e = threadIdx.x; e < ROWS * CPR; e += KRIG_DS_THREADS) {
            int rr = e / CPR, cc = (e % CPR) * VEC;
            int yy = y0 - R + rr, xx = x0 - PAD + cc;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) val = __ldg((const uint4*)(src + (size_t)yy * W + xx));
            *(uint4*)(slot + rr * RP + cc) = val;
        }
    } else {
        for (int e = threadIdx.x; e < ROWS * RP; e += KRIG_DS_THREADS) {
            int rr = e / RP, cc = e % RP;
            int yy = y0 - R + rr, xx = x0 - PAD + cc;
            TI val = TI(0);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) val = src[(size_t)yy * W + xx];
            slot[rr * RP + cc] = val;
        }
    }
}

// Accumulate the stencil of one weight row into the pixels selected by mask.
template <typename TI, int R, int GM1>
__device__ __forceinline__ void ds_accum(typename DsTypes<TI>::TC (&acc)[KRIG_PX][GM1 > 0 ? GM1 : 1],
                                         const TI* lo, const TI* hi, int lrow, int lcol,
                                         const typename DsTypes<TI>::TC* wrow, unsigned mask)
{
    typedef typename DsTypes<TI>::TC TC;
    constexpr int PAD = DsTypes<TI>::PAD;
    constexpr int RP = KRIG_TX + 2 * PAD;
    constexpr int N2R = 2 * R + 1;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const TI* slot = s == 0 ? lo : hi;
#pragma unroll
        for (int dy = -R; dy <= R; ++dy) {
            const TI* rowp = slot + (lrow + R + dy) * RP + PAD + lcol;
            TC a[4], b[4], c[4];
            ld4(rowp - 4, a);
            ld4(rowp, b);
            ld4(rowp + 4, c);
            TC vals[12] = {a[0], a[1], a[2], a[3], b[0], b[1], b[2], b[3], c[0], c[1], c[2], c[3]};
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                TC w[8];
                ldw(wrow + ((s * N2R + (dy + R)) * N2R + (dx + R)) * KRIG_TSLOTS, w);
#pragma unroll
                for (int p = 0; p < KRIG_PX; ++p) {
                    if (!((mask >> p) & 1u)) continue;
                    TC x = vals[4 + p + dx];
#pragma unroll
                    for (int t = 0; t < GM1; ++t) acc[p][t] = fma(w[t], x, acc[p][t]);
                }
            }
        }
    }
}

template <typename TI, int R, int GM1>
__device__ void ds_item(const KrigLaunch& P, int v, int64_t local, TI* sm)
{
    typedef typename DsTypes<TI>::TC TC;
    typedef typename DsTypes<TI>::TO TO;
    constexpr int PAD = DsTypes<TI>::PAD;
    constexpr int RP = KRIG_TX + 2 * PAD;
    constexpr int ROWS = KRIG_TY + 2 * R;
    constexpr int SLOT = ROWS * RP;
    constexpr int NTAP = 2 * (2 * R + 1) * (2 * R + 1);
    const KrigVol& V = P.vol[v];
    const int H = V.H, W = V.W, g = V.g;
    const int64_t plane = (int64_t)H * W;
    const int64_t tiles = (int64_t)V.tiles_x * V.tiles_y;
    const int b = (int)(local / tiles);
    const int rem = (int)(local % tiles);
    const int x0 = (rem % V.tiles_x) * KRIG_TX, y0 = (rem / V.tiles_x) * KRIG_TY;
    const int G = V.n - 1, q = G / V.k, rm = G % V.k;
    const int a0 = b * q + min(b, rm), a1 = (b + 1) * q + min(b + 1, rm);
    const bool last_block = (b == V.k - 1);

    const int lrow = threadIdx.x / (KRIG_TX / KRIG_PX);
    const int lcol = (threadIdx.x % (KRIG_TX / KRIG_PX)) * KRIG_PX;
    const int y = y0 + lrow, xb = x0 + lcol;
    const bool row_in = y < H;
    const int nvalid = min(KRIG_PX, W - xb);
    const bool active = row_in && nvalid > 0;
    const bool vec_out = (W % KRIG_PX == 0) && nvalid == KRIG_PX;
    const bool vec_rows = (W % (16 / (int)sizeof(TI))) == 0;

    const TI* in = (const TI*)P.in[v];
    TO* out = (TO*)P.out[v];
    float* var = P.var[v];
    const TC* wt = (const TC*)(P.ws + V.wtab_off);
    const float* vt = (const float*)(P.ws + V.vtab_off);

    int cy = 0, cxp[KRIG_PX];
    if (active) {
        cy = V.ymap[krig_slot(y, H, R)];
#pragma unroll
        for (int p = 0; p < KRIG_PX; ++p) cxp[p] = V.xmap[krig_slot(p < nvalid ? xb + p : xb, W, R)];
    } else {
#pragma unroll
        for (int p = 0; p < KRIG_PX; ++p) cxp[p] = 0;
    }

    TI* slot0 = sm;
    TI* slot1 = sm + SLOT;
    ds_fill<TI, R>(slot0, in + (size_t)a0 * plane, x0, y0, H, W, vec_rows);
    for (int j = a0; j < a1; ++j) {
        TI* lo = ((j - a0) & 1) ? slot1 : slot0;
        TI* hi = ((j - a0) & 1) ? slot0 : slot1;
        ds_fill<TI, R>(hi, in + (size_t)(j + 1) * plane, x0, y0, H, W, vec_rows);
        __syncthreads();
        if (active) {
            const int64_t pix = (int64_t)y * W + xb;
            // known slice j -> output slice j*g, bit-exact
            {
                TO kv[4];
                const TI* c = lo + (lrow + R) * RP + PAD + lcol;
#pragma unroll
                for (int p = 0; p < 4; ++p) kv[p] = (TO)cvt_out(c[p], V.scale);
                st4<TO>(out + (int64_t)j * g * plane + pix, kv, vec_out, nvalid);
                if (var) {
                    float z4[4] = {0.f, 0.f, 0.f, 0.f};
                    st4<float>(var + (int64_t)j * g * plane + pix, z4, vec_out, nvalid);
                }
                if (last_block && j == a1 - 1) {
                    const TI* ch = hi + (lrow + R) * RP + PAD + lcol;
#pragma unroll
                    for (int p = 0; p < 4; ++p) kv[p] = (TO)cvt_out(ch[p], V.scale);
                    st4<TO>(out + (int64_t)(j + 1) * g * plane + pix, kv, vec_out, nvalid);
                    if (var) {
                        float z4[4] = {0.f, 0.f, 0.f, 0.f};
                        st4<float>(var + (int64_t)(j + 1) * g * plane + pix, z4, vec_out, nvalid);
                    }
                }
            }
            if (GM1 > 0) {
                TC acc[KRIG_PX][GM1 > 0 ? GM1 : 1];
#pragma unroll
                for (int p = 0; p < KRIG_PX; ++p)
#pragma unroll
                    for (int t = 0; t < (GM1 > 0 ? GM1 : 1); ++t) acc[p][t] = TC(0);
                // one pass per distinct x-class among this thread's pixels
                unsigned done = 0;
#pragma unroll 1
                for (int p0 = 0; p0 < KRIG_PX; ++p0) {
                    if ((done >> p0) & 1u) continue;
                    unsigned mask = 0;
#pragma unroll
                    for (int p = 0; p < KRIG_PX; ++p)
                        if (cxp[p] == cxp[p0]) mask |= 1u << p;
                    done |= mask;
                    const TC* wrow = wt + ((int64_t)cy * V.ncx + cxp[p0]) * NTAP * KRIG_TSLOTS;
                    ds_accum<TI, R, GM1>(acc, lo, hi, lrow, lcol, wrow, mask);
                }
#pragma unroll
                for (int t = 0; t < GM1; ++t) {
                    TO o[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p) o[p] = (TO)acc[p][t];
                    st4<TO>(out + ((int64_t)j * g + t + 1) * plane + pix, o, vec_out, nvalid);
                    if (var) {
                        float vv[4];
#pragma unroll
                        for (int p = 0; p < 4; ++p) vv[p] = vt[((int64_t)cy * V.ncx + cxp[p]) * KRIG_TSLOTS + t];
                        st4<float>(var + ((int64_t)j * g + t + 1) * plane + pix, vv, vec_out, nvalid);
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename TI, int R>
__device__ __forceinline__ void ds_dispatch_g(const KrigLaunch& P, int v, int64_t local, TI* sm)
{
    switch (P.vol[v].g) {
    case 1: ds_item<TI, R, 0>(P, v, local, sm); break;
    case 2: ds_item<TI, R, 1>(P, v, local, sm); break;
    case 3: ds_item<TI, R, 2>(P, v, local, sm); break;
    case 4: ds_item<TI, R, 3>(P, v, local, sm); break;
    case 5: ds_item<TI, R, 4>(P, v, local, sm); break;
    case 6: ds_item<TI, R, 5>(P, v, local, sm); break;
    case 7: ds_item<TI, R, 6>(P, v, local, sm); break;
    default: ds_item<TI, R, 7>(P, v, local, sm); break;
    }
}

template <typename TI>
__device__ __forceinline__ void ds_dispatch_r(const KrigLaunch& P, int v, int64_t local, unsigned char* sm)
{
    switch (P.vol[v].r) {
    case 0: ds_dispatch_g<TI, 0>(P, v, local, (TI*)sm); break;
    case 1: ds_dispatch_g<TI, 1>(P, v, local, (TI*)sm); break;
    default: ds_dispatch_g<TI, 2>(P, v, local, (TI*)sm); break;
    }
}

__global__ void __launch_bounds__(KRIG_DS_THREADS) k_ds_apply(const __grid_constant__ KrigLaunch P)
{
    extern __shared__ __align__(16) unsigned char sm[];
    for (int64_t it = blockIdx.x; it < P.n_items; it += gridDim.x) {
        const int v = krig_find_vol(P, it, 0);
        const int64_t local = it - P.vol[v].item_begin;
        switch (P.vol[v].dtype) {
        case KRIG_F64: ds_dispatch_r<double>(P, v, local, sm); break;
        case KRIG_F32: ds_dispatch_r<float>(P, v, local, sm); break;
        default: ds_dispatch_r<uint16_t>(P, v, local, sm); break;
        }
    }
}

static size_t ds_smem_bytes(const KrigLaunch& L)
{
    size_t m = 0;
    for (int v = 0; v < L.n_vols; ++v) {
        const KrigVol& V = L.vol[v];
        size_t esz = V.dtype == KRIG_F64 ? 8 : V.dtype == KRIG_F32 ? 4 : 2;
        size_t pad = V.dtype == KRIG_U16 ? 8 : 4;
        size_t b = 2 * (size_t)(KRIG_TY + 2 * V.r) * (KRIG_TX + 2 * pad) * esz;
        if (b > m) m = b;
    }
    return m;
}

int krig_launch_ds_apply(const KrigLaunch& L, int grid, void* stream)
{
    if (L.n_items == 0) return 0;
    size_t smem = ds_smem_bytes(L);
    if (grid <= 0 || (int64_t)grid > L.n_items) grid = (int)(L.n_items < (1 << 30) ? L.n_items : (1 << 30));
    k_ds_apply<<<grid, KRIG_DS_THREADS, smem, (cudaStream_t)stream>>>(L);
    return (int)cudaGetLastError();
}

int krig_device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}
