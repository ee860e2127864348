// krig_ds_apply.cuh -- stencil apply of the deduplicated-stencil (DS) form.
//
// Every missing voxel (x, y, jg+t) is the weighted sum of the (2r+1)^2
// windows around (x, y) in known slices j and j+1 (Sec. 4.1.2), with the
// weights of its truncation class solved by k_ds_solve.  k_ds_apply walks the
// work items of Algorithm 1: an item is one 64 x 16 in-plane tile of a run of
// consecutive gaps ("chunk") inside one Z sub-block.  The item's known slices
// (tile plus halo) stream through a ring of shared-memory slots filled by the
// TMA engine (completion on an mbarrier), ahead of the compute, so each known
// slice of the chunk is read from memory once.  The item writes its output
// slices -- the bit-exact copy of its known slices (Algorithm 1 step 3) and the
// interpolated ones -- straight to their final offsets (the merge of Sec. 4.2).
//
// Interior pixels (full window) use the D4 symmetry of the interior class:
// the taps of each orbit {same max(|dx|,|dy|), min(|dx|,|dy|)} share one
// weight, so the stencil is applied to orbit sums (6 per slice for r = 2)
// instead of 25 taps; a slice's orbit sums serve both gaps it brackets.
// Pixels within r of the slice border ("frame" pixels) take the general path
// with the full weight row of their own class, in units of 32 handed out by a
// ticket counter to every warp once its slices or items are done.
//
// Items are numbered by input type and stencil shape (the host sorts the
// volumes), so each block walks one contiguous range per shape, round-robin
// across blocks, and every per-item lookup reads a per-block copy of the
// volume table in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "krig_device.cuh"

template <typename TI> struct DsTypes;
template <> struct DsTypes<double> {
    typedef double TC, TO, TW;
    static constexpr int PAD = 4, RP = 72;
};
template <> struct DsTypes<float> {
    typedef float TC, TO;
    typedef unsigned long long TW;
    static constexpr int PAD = 8, RP = 80;
};
template <> struct DsTypes<uint16_t> {
    typedef float TC, TO;
    typedef unsigned long long TW;
    static constexpr int PAD = 8, RP = 96;
};
// TC: arithmetic type; TO: output type; TW: orbit-weight entry in shared memory
// (FP32: the weight twice, the operand of the packed FMAs).  RP (elements per
// shared row) >= TX + 2 PAD; RP * sizeof is 64 mod 128 bytes so the two rows
// read by a quarter warp fall in different banks.

#define DS_CONSUMERS 8                      // consumer warps (tiles)
#define DS_PRODUCER DS_CONSUMERS            // streams the known-slice tiles
#define DS_BLOCK ((DS_CONSUMERS + 1) * 32)  // 9 warps, two blocks per SM
#define DS_WAIT_LIMIT (1u << 22)

// Ring depth per input type.  Slots are released as soon as a slice's orbit
// sums are formed, so a few slices ahead suffice; a shallow ring leaves the
// rest of the SM's 256 KB of L1 / shared memory to the L1 cache (measured: 6
// float slots run the batch and brain stacks 4-9 % faster than 12).
template <typename TI> struct DsStages;
template <> struct DsStages<uint16_t> { static constexpr int S = 10; };
template <> struct DsStages<float> { static constexpr int S = 6; };
template <> struct DsStages<double> { static constexpr int S = 4; };

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// 3-D tiled TMA load of one box into shared memory; completion on the mbarrier.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
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

__device__ __forceinline__ void ldw8(const float* p, float w[8])
{
    float4 a = *(const float4*)p, b = *(const float4*)(p + 4);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}
__device__ __forceinline__ void ldw8(const double* p, double w[8])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double2 a = *(const double2*)(p + 2 * q);
        w[2 * q] = a.x; w[2 * q + 1] = a.y;
    }
}
__device__ __forceinline__ void ldgw8(const float* p, float w[8])
{
    float4 a = __ldg((const float4*)p), b = __ldg((const float4*)(p + 4));
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}
__device__ __forceinline__ void ldgw8(const double* p, double w[8])
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
        for (int q = 0; q < 4; ++q)
            if (q < nvalid) p[q] = v[q];
    }
}

// ---------------------------------------------------------------------------
// Slot fill by warp 0: lane i handles shared row i (tile row + halo).  Rows
// and column ranges outside the slice are zero-filled with ordinary stores
// (they meet zero weights of truncated taps); the rest arrives by bulk copy.
// x0 - PAD and W are multiples of the 16-byte chunk, so every copied segment
// starts and ends on a 16-byte boundary.
// ---------------------------------------------------------------------------
template <typename TI, int R>
__device__ __forceinline__ void ds_issue_fill(TI* slot, uint64_t* bar, const TI* src, int x0, int y0, int H, int W,
                                              int lane)
{
    constexpr int PAD = DsTypes<TI>::PAD, RP = DsTypes<TI>::RP;
    constexpr int ROWS = KRIG_TY + 2 * R;
    constexpr int SPAN = KRIG_TX + 2 * PAD;
    constexpr int VEC = 16 / sizeof(TI);
    const int xs = x0 - PAD;
    const int xa = max(xs, 0), xb = min(xs + SPAN, W);
    const int ya = max(y0 - R, 0), yb = min(y0 + KRIG_TY + R, H);
    const uint32_t row_bytes = (uint32_t)(xb - xa) * sizeof(TI);
    const uint32_t total = row_bytes * (uint32_t)(yb - ya);
    for (int rr = lane; rr < ROWS; rr += 32) {
        const int yy = y0 - R + rr;
        TI* row = slot + rr * RP;
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        if (yy < ya || yy >= yb) {
            for (int c = 0; c < SPAN; c += VEC) *(uint4*)(row + c) = z;
        } else {
            for (int c = 0; c < xa - xs; c += VEC) *(uint4*)(row + c) = z;
            for (int c = xb - xs; c < SPAN; c += VEC) *(uint4*)(row + c) = z;
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(bar, total);
    __syncwarp();
    for (int rr = lane; rr < ROWS; rr += 32) {
        const int yy = y0 - R + rr;
        if (yy >= ya && yy < yb && row_bytes)
            bulk_g2s(slot + rr * RP + (xa - xs), src + (size_t)yy * W + xa, row_bytes, bar);
    }
}

// Plain-load fill by the producer warp for slices whose rows are not
// 16-byte multiples (any W); completion is a plain arrive on the barrier.
template <typename TI, int R>
__device__ __forceinline__ void ds_plain_fill(TI* slot, uint64_t* bar, const TI* src, int x0, int y0, int H, int W,
                                              int lane)
{
    constexpr int PAD = DsTypes<TI>::PAD, RP = DsTypes<TI>::RP;
    constexpr int ROWS = KRIG_TY + 2 * R;
    constexpr int SPAN = KRIG_TX + 2 * PAD;
    for (int e = lane; e < ROWS * SPAN; e += 32) {
        const int rr = e / SPAN, cc = e % SPAN;
        const int yy = y0 - R + rr, xx = x0 - PAD + cc;
        TI val = TI(0);
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) val = src[(size_t)yy * W + xx];
        slot[rr * RP + cc] = val;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
}

// ---------------------------------------------------------------------------
// Per-volume record of the stencil, copied once per block into shared memory
// (the kernel parameter block holds every field, but reads that miss the
// constant cache cost a round trip each; the item and frame loops read these).
// ---------------------------------------------------------------------------
struct DsVolS {
    const void* in;
    void* out;
    float* var;
    const void* mm;                // [k][2] min, max of each sub-block's known voxels, or null (no clamp)
    uint64_t mt, mc, mx;           // multiply-high divisors: tiles, chunks, tiles_x
    int64_t wtab_off, vtab_off, otab_off;
    int32_t item_begin, item_end;  // work items [begin, end)
    int32_t frame_begin, frame_end;  // frame units [begin, end) among the volumes of this input type
    int32_t H, W, n, g;
    int32_t r, dtype, tiles_x, tiles;
    int32_t chunks, chunk, gq, grm;
    int32_t cint, n_frame, frame_units, ncx;
    float scale;
    int8_t xmap[(KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    int8_t ymap[(KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    int8_t pad[10];
};
static_assert(sizeof(DsVolS) % 16 == 0, "DsVolS must keep 16-byte alignment of the table");

__device__ __forceinline__ void ds_fill_vols(const KrigLaunch& P, DsVolS* tab)
{
    for (int v = threadIdx.x; v < P.n_vols; v += blockDim.x) {
        const KrigVol& V = P.vol[v];
        DsVolS s;
        s.in = P.in[v];
        s.out = P.out[v];
        s.var = P.var[v];
        s.mm = P.clamp ? (const void*)(P.ws + V.mm_off) : nullptr;
        s.mt = V.mdiv_tiles;
        s.mc = V.mdiv_chunks;
        s.mx = V.mdiv_tx;
        s.wtab_off = V.wtab_off;
        s.vtab_off = V.vtab_off;
        s.otab_off = V.otab_off;
        s.item_begin = (int32_t)V.item_begin;
        s.item_end = (int32_t)(V.item_begin + (int64_t)V.k * V.chunks * V.tiles_x * V.tiles_y);
        s.frame_begin = (int32_t)V.frame_begin;
        s.frame_end = (int32_t)(V.frame_begin + (int64_t)(V.n - 1) * V.frame_units);
        s.H = V.H;
        s.W = V.W;
        s.n = V.n;
        s.g = V.g;
        s.r = V.r;
        s.dtype = V.dtype;
        s.tiles_x = V.tiles_x;
        s.tiles = V.tiles_x * V.tiles_y;
        s.chunks = V.chunks;
        s.chunk = V.chunk;
        s.gq = V.gq;
        s.grm = V.grm;
        s.cint = V.cint;
        s.n_frame = V.n_frame;
        s.frame_units = V.frame_units;
        s.ncx = V.ncx;
        s.scale = V.scale;
        for (int i = 0; i < (KRIG_RMAX + 1) * (KRIG_RMAX + 1); ++i) {
            s.xmap[i] = V.xmap[i];
            s.ymap[i] = V.ymap[i];
        }
        for (int i = 0; i < 10; ++i) s.pad[i] = 0;
        tab[v] = s;
    }
}

// Dynamic shared memory of k_ds_apply: DS_STAGES ring slots, the full and
// empty barriers, the test barrier, the abort flag and the per-warp "weights
// not yet waited for" flags, the interior orbit weights of every volume and
// the volume table.  Offsets depend on the number of volumes.
extern __shared__ __align__(128) unsigned char ds_smem[];
template <typename TI> struct DsLayout {
    typedef typename DsTypes<TI>::TC TC;
    static constexpr int S = DsStages<TI>::S;
    static constexpr int stride = (KRIG_TY + 2 * KRIG_RMAX) * DsTypes<TI>::RP;  // slot stride, elements
    static constexpr size_t bar_off = (size_t)S * stride * sizeof(TI);
    static constexpr size_t flag_off = bar_off + (2 * S + 1) * sizeof(uint64_t);
    static constexpr size_t ow_off = (flag_off + 4 * (1 + DS_CONSUMERS) + 15) / 16 * 16;
    static constexpr size_t ow_per_vol = 2 * KRIG_NORB * KRIG_TSLOTS * sizeof(typename DsTypes<TI>::TW);
    __host__ __device__ static constexpr size_t vol_off(int nv) { return ow_off + (size_t)nv * ow_per_vol; }
    __host__ __device__ static constexpr size_t bytes(int nv) { return vol_off(nv) + (size_t)nv * sizeof(DsVolS); }
    __device__ static __forceinline__ TI* slots() { return (TI*)ds_smem; }
    __device__ static __forceinline__ uint64_t* full() { return (uint64_t*)(ds_smem + bar_off); }
    __device__ static __forceinline__ uint64_t* empty() { return (uint64_t*)(ds_smem + bar_off) + S; }
    __device__ static __forceinline__ uint64_t* never() { return (uint64_t*)(ds_smem + bar_off) + 2 * S; }
    __device__ static __forceinline__ int* abort_flag() { return (int*)(ds_smem + flag_off); }
    __device__ static __forceinline__ int* pending(int warp) { return (int*)(ds_smem + flag_off) + 1 + warp; }
    __device__ static __forceinline__ typename DsTypes<TI>::TW* ow()
    {
        return (typename DsTypes<TI>::TW*)(ds_smem + ow_off);
    }
    __device__ static __forceinline__ const DsVolS* vols(int nv) { return (const DsVolS*)(ds_smem + vol_off(nv)); }
};

struct DsItem {
    int c0, c1, x0, y0, b;  // gaps [c0, c1), tile origin, Z sub-block
};

// item -> (sub-block b, chunk ch, tile): item = (b * chunks + ch) * tiles + tile,
// divisions by multiply-high.
__device__ __forceinline__ bool ds_decode(const DsVolS& V, int it, DsItem& d)
{
    const uint32_t local = (uint32_t)(it - V.item_begin);
    const uint32_t rest = krig_udiv(local, V.mt), tile = local - rest * (uint32_t)V.tiles;
    const uint32_t bb = krig_udiv(rest, V.mc), ch = rest - bb * (uint32_t)V.chunks;
    const uint32_t ty = krig_udiv(tile, V.mx), tx = tile - ty * (uint32_t)V.tiles_x;
    const int b = (int)bb;
    const int a0 = b * V.gq + min(b, V.grm), a1 = (b + 1) * V.gq + min(b + 1, V.grm);
    d.b = b;
    d.c0 = a0 + (int)ch * V.chunk;
    d.c1 = min(d.c0 + V.chunk, a1);
    d.x0 = (int)tx * KRIG_TX;
    d.y0 = (int)ty * KRIG_TY;
    return d.c0 < d.c1;
}

// Stencil shape of a volume: (r, g).
__device__ __forceinline__ int ds_shape(const DsVolS& V) { return V.r * 8 + V.g - 1; }

// The run of volumes [k, *k_end) in item order that share the input type and
// shape of ds_order[k]; false if ds_order[k] is of another input type.
__device__ __forceinline__ bool ds_run(const int8_t* order, const DsVolS* tab, int nv, int dtype, int k, int* k_end)
{
    const DsVolS& V = tab[order[k]];
    int e = k + 1;
    while (e < nv && tab[order[e]].dtype == V.dtype && ds_shape(tab[order[e]]) == ds_shape(V)) ++e;
    *k_end = e;
    return V.dtype == dtype;
}

// First item >= lo of this block's round-robin sequence it = blockIdx.x (mod grid).
__device__ __forceinline__ int ds_first_item(int lo)
{
    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    return lo + (((b - lo) % G) + G) % G;
}

// ---------------------------------------------------------------------------
// Interior path.  A thread owns four consecutive pixels, taken as two pixel
// pairs; every orbit sum, partial sum and output of a pair is one packed value
// (FP32: a 64-bit register pair and the f32x2 instructions, each half rounding
// as the scalar instruction; FP64: two doubles), so the arithmetic needs no
// operand shuffling.  The D4 orbit sums of a known slice ({same
// max(|dx|,|dy|), min(|dx|,|dy|)}: 1, 3, 6 for r = 0, 1, 2) are formed once per
// slice.  The slice then completes the gap below it as its upper slice, from
// the partial sums over the lower slice kept since that one arrived, and
// starts the gap above it as its lower slice (new partial sums); between
// slices a thread keeps g - 1 partial sums per pixel pair, not a slice of
// orbit sums.  Every output is sum_s sum_o w[s][o][t] O_s[o] accumulated in
// the order s = lower, upper and o ascending, by fused multiply-adds.
// ---------------------------------------------------------------------------
template <int R> struct DsNO { static constexpr int N = R == 0 ? 1 : (R == 1 ? 3 : 6); };
template <int GM1> struct DsGP { static constexpr int N = GM1 > 0 ? GM1 : 1; };  // partial sums per pixel pair

// One shared row around the thread's pixels: columns lcol-4 .. lcol+7 (pixel
// p at column 4 + p) as six column pairs; only the pairs a window of half
// width R reaches are loaded.
template <typename TI, int R>
__device__ __forceinline__ void ds_row_pairs(const TI* rowp, Px2<typename DsTypes<TI>::TC> (&c)[6])
{
    typedef typename DsTypes<TI>::TC TC;
    TC v[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) v[i] = TC(0);
    if (R > 0) ld4(rowp - 4, v);
    ld4(rowp, v + 4);
    if (R > 0) ld4(rowp + 4, v + 8);
#pragma unroll
    for (int i = 0; i < 6; ++i) c[i] = Px2<TC>::of(v[2 * i], v[2 * i + 1]);
}

// D4 orbit sums of one known slice at the thread's two pixel pairs:
//   o0 = c, o1 = (c(+-1, 0)) + (c(0, +-1)), o2 = c(+-1, +-1),
//   o3 = (c(+-2, 0)) + (c(0, +-2)), o4 = (c(+-2, +-1)) + (c(+-1, +-2)), o5 = c(+-2, +-2),
// with each parenthesised pair of taps added first, rows +-d summed before the
// column shifts.
template <typename TI, int R>
__device__ __forceinline__ void ds_orbits(const TI* slot, int lrow, int lcol,
                                          Px2<typename DsTypes<TI>::TC> (&O)[2][DsNO<R>::N])
{
    typedef typename DsTypes<TI>::TC TC;
    constexpr int PAD = DsTypes<TI>::PAD, RP = DsTypes<TI>::RP;
    const TI* base = slot + (lrow + R) * RP + PAD + lcol;
    Px2<TC> c0[6];
    ds_row_pairs<TI, R>(base, c0);
#pragma unroll
    for (int k = 0; k < 2; ++k) O[k][0] = c0[2 + k];
    if (R >= 1) {
        Px2<TC> a1[6], b[6];
        ds_row_pairs<TI, R>(base - RP, a1);
        ds_row_pairs<TI, R>(base + RP, b);
#pragma unroll
        for (int i = 0; i < 6; ++i) a1[i] = a1[i] + b[i];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            O[k][1] = px_s1(c0, k) + a1[2 + k];
            O[k][2] = px_s1(a1, k);
        }
        if (R >= 2) {
            Px2<TC> a2[6];
            ds_row_pairs<TI, R>(base - 2 * RP, a2);
            ds_row_pairs<TI, R>(base + 2 * RP, b);
#pragma unroll
            for (int i = 0; i < 6; ++i) a2[i] = a2[i] + b[i];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                O[k][3] = px_s2(c0, k) + a2[2 + k];
                O[k][4] = px_s2(a1, k) + px_s1(a2, k);
                O[k][5] = px_s2(a2, k);
            }
        }
    }
}

// Per-item constants of a consumer thread.
template <typename TI>
struct DsCtx {
    typename DsTypes<TI>::TO* out;  // output at this thread's first pixel, slice 0
    float* var;                     // variance likewise, or null
    const float* vt;                // variance row of the interior class
    int64_t plane;                  // H * W
    int g, jlast;                   // Z factor; gap index whose upper slice is the last one
    float scale;
    int nvalid, plo, phi;           // valid pixels of the four; interior ones [plo, phi)
    bool mine, vec_out, inner, full;
    bool clamp;                     // clamp the estimates to [lo, hi], the sub-block's known range
    typename DsTypes<TI>::TC lo, hi;
};

template <typename TI, int R>
__device__ __forceinline__ DsCtx<TI> ds_ctx(const DsVolS& V, const unsigned char* ws, const DsItem& d, int lrow,
                                            int lcol, bool dry)
{
    typedef typename DsTypes<TI>::TO TO;
    DsCtx<TI> c;
    const int H = V.H, W = V.W;
    const int y = d.y0 + lrow, xb = d.x0 + lcol;
    c.plane = (int64_t)H * W;
    c.g = V.g;
    c.jlast = V.n - 2;
    c.scale = V.scale;
    c.nvalid = min(KRIG_PX, W - xb);
    c.mine = y < H && c.nvalid > 0;
    c.vec_out = (W % KRIG_PX == 0) && c.nvalid == KRIG_PX;
    const int64_t pix = c.mine ? (int64_t)y * W + xb : 0;
    c.out = (TO*)V.out + pix;
    c.var = (dry || !V.var) ? nullptr : V.var + pix;
    c.vt = (const float*)(ws + V.vtab_off) + (int64_t)max(V.cint, 0) * KRIG_TSLOTS;
    // interior pixels of the four: rows y in [R, H-1-R], x in [R, W-1-R]
    c.plo = max(0, R - xb);
    c.phi = min(c.nvalid, W - R - xb);
    c.inner = c.mine && V.cint >= 0 && y >= R && y <= H - 1 - R && c.plo < c.phi;
    c.full = c.vec_out && c.plo == 0 && c.phi == KRIG_PX;
    c.clamp = V.mm != nullptr;
    c.lo = c.hi = 0;
    if (c.clamp) {
        const typename DsTypes<TI>::TC* mm = (const typename DsTypes<TI>::TC*)V.mm + 2 * d.b;
        c.lo = mm[0];
        c.hi = mm[1];
    }
    return c;
}

// Known slice -> its output slice, bit-exact (u16: float32(u) * scale); o: the
// slice's values at the two pixel pairs.
template <typename TI>
__device__ __forceinline__ void ds_passthrough(const DsCtx<TI>& c, int64_t off, Px2<typename DsTypes<TI>::TC> o0,
                                               Px2<typename DsTypes<TI>::TC> o1)
{
    typedef typename DsTypes<TI>::TO TO;
    TO kv[4] = {(TO)o0.x(), (TO)o0.y(), (TO)o1.x(), (TO)o1.y()};
    if (sizeof(TI) == 2) {
#pragma unroll
        for (int p = 0; p < 4; ++p) kv[p] = (TO)__fmul_rn((float)kv[p], c.scale);
    }
    st4<TO>(c.out + off, kv, c.vec_out, c.nvalid);
    if (c.var) {
        const float z4[4] = {0.f, 0.f, 0.f, 0.f};
        st4<float>(c.var + off, z4, c.vec_out, c.nvalid);
    }
}

// acc[t][k] += sum_o w[o][t] O[k][o] for every target t (o ascending): w is one
// slice's [NORB][8] block of the orbit-weight table; the FP32 table is read two
// targets ((w_t, w_t), (w_t+1, w_t+1)) per 16-byte load.
template <typename TI, int NO, int GM1>
__device__ __forceinline__ void ds_accum_slice(Px2<typename DsTypes<TI>::TC> (&acc)[DsGP<GM1>::N][2],
                                               const Px2<typename DsTypes<TI>::TC> (&O)[2][NO],
                                               const typename DsTypes<TI>::TW* w)
{
    typedef typename DsTypes<TI>::TC TC;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
#pragma unroll
        for (int t = 0; t < GM1; t += 2) {
            Px2<TC> wa, wb;
            if constexpr (sizeof(TC) == 4) {
                const ulonglong2 q = *(const ulonglong2*)(w + o * KRIG_TSLOTS + t);
                wa = px_w(q.x);
                wb = px_w(q.y);
            } else {
                const double2 q = *(const double2*)(w + o * KRIG_TSLOTS + t);
                wa = px_w(q.x);
                wb = px_w(q.y);
            }
            px_fma(acc[t][0], wa, O[0][o]);
            px_fma(acc[t][1], wa, O[1][o]);
            if (t + 1 < GM1) {
                px_fma(acc[t + 1][0], wb, O[0][o]);
                px_fma(acc[t + 1][1], wb, O[1][o]);
            }
        }
    }
}

// Interpolated output slice (target t + 1) at offset off for the interior
// pixels of the four (and their kriging variance); u0, u1: the two pixel pairs.
template <typename TI>
__device__ __forceinline__ void ds_store_t(const DsCtx<TI>& c, int64_t off, int t, Px2<typename DsTypes<TI>::TC> u0,
                                           Px2<typename DsTypes<TI>::TC> u1)
{
    typedef typename DsTypes<TI>::TO TO;
    typedef typename DsTypes<TI>::TC TC;
    TC v[4] = {u0.x(), u0.y(), u1.x(), u1.y()};
    if (c.clamp) {
#pragma unroll
        for (int p = 0; p < 4; ++p)  // comparisons keep a NaN (singular system) a NaN
            v[p] = v[p] < c.lo ? c.lo : (v[p] > c.hi ? c.hi : v[p]);
    }
    if (c.full) {
        TO o[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) o[p] = (TO)v[p];
        st4<TO>(c.out + off, o, true, 4);
    } else {
#pragma unroll
        for (int p = 0; p < 4; ++p)
            if (p >= c.plo && p < c.phi) c.out[off + p] = (TO)v[p];
    }
    if (c.var) {
        const float vv = c.vt[t];
        if (c.full) {
            const float v4[4] = {vv, vv, vv, vv};
            st4<float>(c.var + off, v4, true, 4);
        } else {
            for (int p = c.plo; p < c.phi; ++p) c.var[off + p] = vv;
        }
    }
}

// One item for one consumer warp: its 8 x 16 pixel block of the tile, every
// gap of the item's chunk.  Each known slice's orbit sums are formed right
// after its slot fills, and the slot is released at once.  dry: warm-up pass
// over the first gap while the class solve may still run, with no release
// (the slots stay full for the real pass); its stores, from weights not yet
// final, go to the same addresses as the real pass's, which follows in the
// same thread and overwrites them.  ow: the volume's orbit-weight table
// [2][NORB][8] in shared memory.  Returns false if a wait gave up.
template <typename TI, int R, int GM1>
__device__ __forceinline__ bool ds_item(const DsCtx<TI>& c, const DsItem& d, int q, int lrow, int lcol, int lane,
                                        const typename DsTypes<TI>::TW* ow, bool dry)
{
    typedef typename DsTypes<TI>::TC TC;
    constexpr int S = DsStages<TI>::S;
    constexpr int NO = DsNO<R>::N;
    constexpr int GP = DsGP<GM1>::N;
    TI* slots = DsLayout<TI>::slots();
    uint64_t* full = DsLayout<TI>::full();
    uint64_t* empty = DsLayout<TI>::empty();
    constexpr int stride = DsLayout<TI>::stride;
    const int nsl = dry ? 2 : d.c1 - d.c0 + 1;  // warm-up: the first gap only
    const bool fma_px = GM1 > 0 && c.inner;
    // partial sums over the lower slice of the current gap (defined from the
    // start: a conditionally assigned array is kept in local memory)
    Px2<TC> L[GP][2];
#pragma unroll
    for (int t = 0; t < GP; ++t) L[t][0] = L[t][1] = Px2<TC>::zero();
    for (int m = 0; m < nsl; ++m) {
        const int j = d.c0 + m, qs = q + m;  // slice j
        if (!mbar_wait(&full[qs % S], (qs / S) & 1, DS_WAIT_LIMIT)) return false;
        Px2<TC> O[2][NO];
        ds_orbits<TI, R>(slots + (qs % S) * stride, lrow, lcol, O);
        __syncwarp();
        if (lane == 0 && !dry) mbar_arrive(&empty[qs % S]);
        const int64_t jg = (int64_t)j * c.g * c.plane;  // output offset of slice j
        // slices c0 .. c1-1 are the lower slices of this item's gaps; the last
        // slice of the volume is passed through by the item of the last gap
        if (c.mine && (m + 1 < nsl || j - 1 == c.jlast)) ds_passthrough<TI>(c, jg, O[0][0], O[1][0]);
        if constexpr (GM1 > 0) {
            if (fma_px) {
                if (m > 0) {
                    // upper slice of gap j - 1: complete its targets in place (the
                    // chains of all targets are independent), then store them
                    ds_accum_slice<TI, NO, GM1>(L, O, ow + KRIG_NORB * KRIG_TSLOTS);
                    int64_t off = jg - (int64_t)(c.g - 1) * c.plane;  // target 1 of gap j - 1
#pragma unroll
                    for (int t = 0; t < GM1; ++t, off += c.plane) ds_store_t<TI>(c, off, t, L[t][0], L[t][1]);
                }
                if (m + 1 < nsl) {
                    // lower slice of gap j: its partial sums
#pragma unroll
                    for (int t = 0; t < GM1; ++t) L[t][0] = L[t][1] = Px2<TC>::zero();
                    ds_accum_slice<TI, NO, GM1>(L, O, ow);
                }
            }
        }
    }
    return true;
}

// The class solve may still be running (programmatic dependent launch): wait
// for it to complete, then copy the interior orbit weights of all volumes,
// now final, into shared memory; a named barrier over the consumer warps only
// (the producer runs on).  Every consumer warp calls this exactly once: before
// its first real item, or after its last run if it had none.
template <typename TI>
__device__ __noinline__ void ds_weights_ready(const unsigned char* ws, int nv, int dtype)
{
    typedef typename DsTypes<TI>::TC TC;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    typename DsTypes<TI>::TW* owsm = DsLayout<TI>::ow();
    const DsVolS* tab = DsLayout<TI>::vols(nv);
    constexpr int NW = 2 * KRIG_NORB * KRIG_TSLOTS;
    for (int e = threadIdx.x; e < nv * NW; e += DS_CONSUMERS * 32) {
        const DsVolS& Vv = tab[e / NW];
        const TC w = (Vv.dtype == dtype && Vv.cint >= 0) ? ((const TC*)(ws + Vv.otab_off))[e % NW] : TC(0);
        if constexpr (sizeof(TC) == 4) owsm[e] = pk2(w, w);
        else owsm[e] = w;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(DS_CONSUMERS * 32) : "memory");
}

struct DsRunArgs {
    const unsigned char* ws;
    uint32_t* status;
    int nv, k0, k1, warp, lane;
};

// All items of one run (volumes order[k0..k1), one shape) for this block's
// consumer warp; returns the slice sequence number after them, or -1 after a
// wait that gave up.  One non-inlined instance per shape, so the call (and
// its register saves) happens once per run, not once per item.
template <typename TI, int R, int GM1>
__device__ __noinline__ int ds_run_shape(const DsRunArgs a, const int8_t* order, int q)
{
    typedef typename DsTypes<TI>::TC TC;
    const int dtype = sizeof(TI) == 8 ? KRIG_F64 : sizeof(TI) == 4 ? KRIG_F32 : KRIG_U16;
    const DsVolS* tab = DsLayout<TI>::vols(a.nv);
    int* pending = DsLayout<TI>::pending(a.warp);
    const int lrow = (a.warp >> 2) * 8 + (a.lane >> 2);
    const int lcol = (a.warp & 3) * 16 + (a.lane & 3) * 4;
    int k = a.k0;
    const int hi = tab[order[a.k1 - 1]].item_end;
    for (int it = ds_first_item(tab[order[a.k0]].item_begin); it < hi; it += gridDim.x) {
        while (it >= tab[order[k]].item_end) ++k;
        const int v = order[k];
        const DsVolS& V = tab[v];
        DsItem d;
        if (!ds_decode(V, it, d)) continue;
        if (*(volatile int*)DsLayout<TI>::abort_flag()) return -1;
        const typename DsTypes<TI>::TW* ow = DsLayout<TI>::ow() + v * (2 * KRIG_NORB * KRIG_TSLOTS);
        // First item of the warp: a warm-up pass over its first gap (the same code,
        // no stores) while the class solve may still run, so the consumer code is
        // cached when the weights arrive; only then the wait (ds_weights_ready).
        for (int pass = *pending ? 0 : 1; pass < 2; ++pass) {
            const bool dry = pass == 0;
            if (!dry && *pending) {
                ds_weights_ready<TI>(a.ws, a.nv, dtype);
                *pending = 0;
            }
            const DsCtx<TI> c = ds_ctx<TI, R>(V, a.ws, d, lrow, lcol, dry);
            if (!ds_item<TI, R, GM1>(c, d, q, lrow, lcol, a.lane, ow, dry)) return -1;
        }
        q += d.c1 - d.c0 + 1;
    }
    return q;
}

template <typename TI, int R>
__device__ __forceinline__ int ds_run_g(int g, const DsRunArgs& a, const int8_t* order, int q)
{
    switch (g) {
    case 1: return ds_run_shape<TI, R, 0>(a, order, q);
    case 2: return ds_run_shape<TI, R, 1>(a, order, q);
    case 3: return ds_run_shape<TI, R, 2>(a, order, q);
    case 4: return ds_run_shape<TI, R, 3>(a, order, q);
    case 5: return ds_run_shape<TI, R, 4>(a, order, q);
    case 6: return ds_run_shape<TI, R, 5>(a, order, q);
    case 7: return ds_run_shape<TI, R, 6>(a, order, q);
    default: return ds_run_shape<TI, R, 7>(a, order, q);
    }
}

// ---------------------------------------------------------------------------
// Frame units: 32 frame pixels (within r of the slice border) of one gap, one
// lane each, through the full weight row of the pixel's own truncation class.
// Tap coordinates are clamped into the slice and truncated taps carry zero
// weight in the class row, so every load is independent and in flight at once.
// Units are handed out by a ticket counter to every warp of the block once it is
// done with its slices (producer) or items (consumers).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ds_frame_pixel(const DsVolS& V, int f, int* x, int* y)
{
    const int r = V.r, W = V.W, H = V.H;
    if (V.cint < 0) {
        *x = f % W;
        *y = f / W;
    } else if (f < r * W) {
        *x = f % W;
        *y = f / W;
    } else if (f < 2 * r * W) {
        f -= r * W;
        *x = f % W;
        *y = H - r + f / W;
    } else {
        f -= 2 * r * W;
        const int c = f % (2 * r);
        *y = r + f / (2 * r);
        *x = c < r ? c : W - 2 * r + c;
    }
}

template <typename TI, int R, int GM1>
__device__ __noinline__ void ds_frame_unit(const DsVolS& V, const unsigned char* ws, int j, int f0, int lane)
{
    typedef typename DsTypes<TI>::TC TC;
    typedef typename DsTypes<TI>::TO TO;
    constexpr int N2R = 2 * R + 1, NTAP = 2 * N2R * N2R;
    const int f = f0 + lane;
    if (f >= V.n_frame) return;
    int x, y;
    ds_frame_pixel(V, f, &x, &y);
    const int W = V.W, H = V.H, g = V.g;
    const int64_t plane = (int64_t)H * W;
    const int cy = V.ymap[krig_slot(y, H, R)], cx = V.xmap[krig_slot(x, W, R)];
    const TC* wrow = (const TC*)(ws + V.wtab_off) + ((int64_t)cy * V.ncx + cx) * NTAP * KRIG_TSLOTS;
    const TI* in = (const TI*)V.in + (size_t)j * plane;
    TC z[NTAP];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int dy = -R; dy <= R; ++dy)
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                const int yy = min(max(y + dy, 0), H - 1), xx = min(max(x + dx, 0), W - 1);
                z[(s * N2R + dy + R) * N2R + dx + R] = (TC)__ldg(in + (size_t)s * plane + (size_t)yy * W + xx);
            }
    TC acc[GM1];
#pragma unroll
    for (int t = 0; t < GM1; ++t) acc[t] = TC(0);
#pragma unroll
    for (int k = 0; k < NTAP; ++k) {
        TC w[8];
        if constexpr (sizeof(TC) == 4) {
            float4 a = __ldg((const float4*)(wrow + k * KRIG_TSLOTS));
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
            if (GM1 > 4) {
                float4 b = __ldg((const float4*)(wrow + k * KRIG_TSLOTS + 4));
                w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < (GM1 + 1) / 2; ++q) {
                double2 a = __ldg((const double2*)(wrow + k * KRIG_TSLOTS + 2 * q));
                w[2 * q] = a.x;
                w[2 * q + 1] = a.y;
            }
        }
#pragma unroll
        for (int t = 0; t < GM1; ++t) acc[t] = fma(w[t], z[k], acc[t]);
    }
    if (V.mm) {  // the gap's sub-block: the first grm blocks have gq + 1 gaps
        const int big = V.grm * (V.gq + 1);
        const int b = j < big ? j / (V.gq + 1) : V.grm + (j - big) / V.gq;
        const TC* mm = (const TC*)V.mm + 2 * b;
#pragma unroll
        for (int t = 0; t < GM1; ++t) acc[t] = acc[t] < mm[0] ? mm[0] : (acc[t] > mm[1] ? mm[1] : acc[t]);
    }
    TO* out = (TO*)V.out;
    float* var = V.var;
    const float* vt = (const float*)(ws + V.vtab_off) + ((int64_t)cy * V.ncx + cx) * KRIG_TSLOTS;
    const int64_t pix = (int64_t)y * W + x;
#pragma unroll
    for (int t = 0; t < GM1; ++t) {
        out[((int64_t)j * g + t + 1) * plane + pix] = (TO)acc[t];
        if (var) var[((int64_t)j * g + t + 1) * plane + pix] = vt[t];
    }
}

template <typename TI, int GM1>
__device__ __forceinline__ void ds_frame_r(const DsVolS& V, const unsigned char* ws, int j, int f0, int lane)
{
    switch (V.r) {
    case 0: ds_frame_unit<TI, 0, GM1>(V, ws, j, f0, lane); break;
    case 1: ds_frame_unit<TI, 1, GM1>(V, ws, j, f0, lane); break;
    default: ds_frame_unit<TI, 2, GM1>(V, ws, j, f0, lane); break;
    }
}

template <typename TI>
__device__ __noinline__ void ds_frames(const unsigned char* ws, int nv, int dtype, int total, int lane)
{
    const DsVolS* tab = DsLayout<TI>::vols(nv);
    unsigned* ticket = (unsigned*)(ws + KRIG_CTRL_FRAME_NEXT) + dtype;
    int v = 0;
    for (;;) {
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(ticket, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= total) return;
        // the volume of this input type whose frame units contain u (tickets rise, so search on from the last)
        if (!(tab[v].dtype == dtype && u >= tab[v].frame_begin && u < tab[v].frame_end)) {
            v = 0;
            while (v < nv && !(tab[v].dtype == dtype && u >= tab[v].frame_begin && u < tab[v].frame_end)) ++v;
            if (v >= nv) return;  // cannot happen: the units of this type are numbered contiguously
        }
        const DsVolS& V = tab[v];
        const int lu = u - V.frame_begin;
        const int j = lu / V.frame_units;
        const int f0 = (lu - j * V.frame_units) * 32;
        switch (V.g) {
        case 2: ds_frame_r<TI, 1>(V, ws, j, f0, lane); break;
        case 3: ds_frame_r<TI, 2>(V, ws, j, f0, lane); break;
        case 4: ds_frame_r<TI, 3>(V, ws, j, f0, lane); break;
        case 5: ds_frame_r<TI, 4>(V, ws, j, f0, lane); break;
        case 6: ds_frame_r<TI, 5>(V, ws, j, f0, lane); break;
        case 7: ds_frame_r<TI, 6>(V, ws, j, f0, lane); break;
        case 8: ds_frame_r<TI, 7>(V, ws, j, f0, lane); break;
        default: break;  // g = 1: no frame units
        }
    }
}

// ---------------------------------------------------------------------------
// Producer: streams every known slice of the block's items, in the consumers'
// order, into the ring.
// ---------------------------------------------------------------------------
template <typename TI>
__device__ __forceinline__ void ds_produce_slice(const DsVolS& V, const DsItem& d, int s, TI* slot, uint64_t* bar,
                                                 int lane, const CUtensorMap* map)
{
    if (map) {
        // one tensor-map request per slice tile; rows and columns outside the
        // stack arrive as zeros (they meet zero weights of truncated taps)
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(DsTypes<TI>::RP * (KRIG_TY + 2 * V.r) * sizeof(TI));
            mbar_arrive_expect_tx(bar, bytes);
            tma_load_3d(slot, map, d.x0 - DsTypes<TI>::PAD, d.y0 - V.r, s, bar);
        }
        __syncwarp();
        return;
    }
    const int64_t plane = (int64_t)V.H * V.W;
    const TI* src = (const TI*)V.in + (size_t)s * plane;
    const bool bulk = (V.W % (16 / (int)sizeof(TI))) == 0;
    switch (V.r) {
    case 0:
        if (bulk) ds_issue_fill<TI, 0>(slot, bar, src, d.x0, d.y0, V.H, V.W, lane);
        else ds_plain_fill<TI, 0>(slot, bar, src, d.x0, d.y0, V.H, V.W, lane);
        break;
    case 1:
        if (bulk) ds_issue_fill<TI, 1>(slot, bar, src, d.x0, d.y0, V.H, V.W, lane);
        else ds_plain_fill<TI, 1>(slot, bar, src, d.x0, d.y0, V.H, V.W, lane);
        break;
    default:
        if (bulk) ds_issue_fill<TI, 2>(slot, bar, src, d.x0, d.y0, V.H, V.W, lane);
        else ds_plain_fill<TI, 2>(slot, bar, src, d.x0, d.y0, V.H, V.W, lane);
        break;
    }
}

template <typename TI>
__device__ __noinline__ void ds_producer(const DsTma& T, const int8_t* order, uint32_t* status, int nv, int lane)
{
    constexpr int S = DsStages<TI>::S;
    constexpr int stride = DsLayout<TI>::stride;
    const int dtype = sizeof(TI) == 8 ? KRIG_F64 : sizeof(TI) == 4 ? KRIG_F32 : KRIG_U16;
    const DsVolS* tab = DsLayout<TI>::vols(nv);
    TI* slots = DsLayout<TI>::slots();
    uint64_t* full = DsLayout<TI>::full();
    uint64_t* empty = DsLayout<TI>::empty();
    int* abort = DsLayout<TI>::abort_flag();
    int q = 0;
    bool ok = true;
    for (int k0 = 0, k1 = 0; k0 < nv && ok; k0 = k1) {
        if (!ds_run(order, tab, nv, dtype, k0, &k1)) continue;
        int k = k0;
        const int hi = tab[order[k1 - 1]].item_end;
        for (int it = ds_first_item(tab[order[k0]].item_begin); it < hi && ok; it += gridDim.x) {
            while (it >= tab[order[k]].item_end) ++k;
            const int v = order[k];
            const DsVolS& V = tab[v];
            DsItem d;
            if (!ds_decode(V, it, d)) continue;
            const CUtensorMap* map = (v < KRIG_TMA_VOLS && T.valid[v]) ? &T.tm[v] : nullptr;
            for (int s = d.c0; s <= d.c1; ++s, ++q) {
                const int slot = q % S;
                if (q >= S && !mbar_wait(&empty[slot], ((q / S) - 1) & 1, DS_WAIT_LIMIT)) {
                    ok = false;
                    break;
                }
                if (*(volatile int*)abort) {
                    ok = false;
                    break;
                }
                fence_proxy_async_smem();
                ds_produce_slice<TI>(V, d, s, slots + slot * stride, &full[slot], lane, map);
            }
        }
    }
    if (!ok) {
        if (lane == 0) {
            krig_set_status(status, KRIG_DEV_TIMEOUT);
            atomicExch(abort, 1);
        }
        // bounded wait for the copies still in flight (the last S issued)
        for (int qq = max(0, q - S); qq < q; ++qq) mbar_wait(&full[qq % S], (qq / S) & 1, DS_WAIT_LIMIT);
    }
}

// One kernel per input type (compiled in separate translation units); volumes
// of another type are skipped run by run.
template <typename TI>
__global__ void __launch_bounds__(DS_BLOCK, 2) k_ds_apply(const __grid_constant__ KrigLaunch P,
                                                          const __grid_constant__ DsTma T)
{
    constexpr int S = DsStages<TI>::S;
    const int dtype = sizeof(TI) == 8 ? KRIG_F64 : sizeof(TI) == 4 ? KRIG_F32 : KRIG_U16;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nv = P.n_vols;
    if (tid < S) {
        mbar_init(&DsLayout<TI>::full()[tid], 1);
        mbar_init(&DsLayout<TI>::empty()[tid], DS_CONSUMERS);
    }
    if (tid == 0) {
        mbar_init(DsLayout<TI>::never(), 1);
        *DsLayout<TI>::abort_flag() = 0;
    }
    if (tid < DS_CONSUMERS) *DsLayout<TI>::pending(tid) = 1;
    ds_fill_vols(P, (DsVolS*)DsLayout<TI>::vols(nv));
    fence_proxy_async_smem();
    __syncthreads();
    if (warp == DS_PRODUCER) {
        ds_producer<TI>(T, P.ds_order, P.status, nv, lane);
        // then border pixels beside the consumers, once the class solve has completed
        // (programmatic dependent launch: it may still be running)
        asm volatile("griddepcontrol.wait;" ::: "memory");
        ds_frames<TI>(P.ws, nv, dtype, P.ds_frame_units[dtype], lane);
        return;
    }
    // ---------------- consumer warps
    if (P.fault_timeout && blockIdx.x == 0 && warp == 0) {
        // test hook: wait on a barrier nothing completes; the bounded wait gives up
        if (!mbar_wait(DsLayout<TI>::never(), 0, 1u << 12) && lane == 0) {
            krig_set_status(P.status, KRIG_DEV_TIMEOUT);
            atomicExch(DsLayout<TI>::abort_flag(), 1);
        }
    }
    const DsVolS* tab = DsLayout<TI>::vols(nv);
    int q = 0;
    DsRunArgs a{P.ws, P.status, nv, 0, 0, warp, lane};
    for (int k0 = 0, k1 = 0; k0 < nv && q >= 0; k0 = k1) {
        if (!ds_run(P.ds_order, tab, nv, dtype, k0, &k1)) continue;
        const DsVolS& V = tab[P.ds_order[k0]];
        a.k0 = k0;
        a.k1 = k1;
        if (V.r == 0) q = ds_run_g<TI, 0>(V.g, a, P.ds_order, q);
        else if (V.r == 1) q = ds_run_g<TI, 1>(V.g, a, P.ds_order, q);
        else q = ds_run_g<TI, 2>(V.g, a, P.ds_order, q);
    }
    if (q < 0) {
        if (lane == 0) {
            krig_set_status(P.status, KRIG_DEV_TIMEOUT);
            atomicExch(DsLayout<TI>::abort_flag(), 1);
        }
    }
    if (*DsLayout<TI>::pending(warp)) ds_weights_ready<TI>(P.ws, nv, dtype);  // no item: still one arrival
    ds_frames<TI>(P.ws, nv, dtype, P.ds_frame_units[dtype], lane);
}

template <typename TI>
int krig_launch_ds_apply_t(const KrigLaunch& L, const DsTma& T, cudaStream_t st)
{
    const int dtype = sizeof(TI) == 8 ? KRIG_F64 : sizeof(TI) == 4 ? KRIG_F32 : KRIG_U16;
    bool any = false;
    for (int v = 0; v < L.n_vols; ++v) any = any || L.vol[v].dtype == dtype;
    if (!any) return 0;
    const size_t smem = DsLayout<TI>::bytes(L.n_vols);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_ds_apply<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ds_apply<TI>, DS_BLOCK, smem);
    if (e != cudaSuccess) return (int)e;
    const int sms = krig_device_sm_count();
    if (L.ds_blocks_per_sm > 0 && L.ds_blocks_per_sm < per_sm) per_sm = L.ds_blocks_per_sm;
    int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    if (grid > L.n_items) grid = L.n_items;
    if (grid < 1) grid = 1;
    // programmatic dependent launch: this grid may start while the class
    // solve before it on the stream is still running
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(DS_BLOCK);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_ds_apply<TI>, L, T);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaGetLastError();
}
