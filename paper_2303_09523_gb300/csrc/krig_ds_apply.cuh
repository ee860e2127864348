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
template <> struct DsTypes<double> { typedef double TC; typedef double TO; static constexpr int PAD = 4, RP = 72; };
template <> struct DsTypes<float> { typedef float TC; typedef float TO; static constexpr int PAD = 8, RP = 80; };
template <> struct DsTypes<uint16_t> { typedef float TC; typedef float TO; static constexpr int PAD = 8, RP = 96; };
// RP (elements per shared row) >= TX + 2 PAD; RP * sizeof is 64 mod 128 bytes so the
// two rows read by a quarter warp fall in different banks.

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
    static constexpr size_t ow_per_vol = 2 * KRIG_NORB * KRIG_TSLOTS * sizeof(TC);
    __host__ __device__ static constexpr size_t vol_off(int nv) { return ow_off + (size_t)nv * ow_per_vol; }
    // per consumer thread, the orbit sums of the previous slice when they do not stay in
    // registers (ds_lo_smem): [NORB][256 threads][4 pixels]
    __host__ __device__ static constexpr size_t orb_off(int nv)
    {
        return (vol_off(nv) + (size_t)nv * sizeof(DsVolS) + 15) / 16 * 16;
    }
    static constexpr size_t orb_bytes = (size_t)KRIG_NORB * DS_CONSUMERS * 32 * KRIG_PX * sizeof(TC);
    __host__ __device__ static constexpr size_t bytes(int nv) { return orb_off(nv) + orb_bytes; }
    __device__ static __forceinline__ TC* orb(int nv) { return (TC*)(ds_smem + orb_off(nv)); }
    __device__ static __forceinline__ TI* slots() { return (TI*)ds_smem; }
    __device__ static __forceinline__ uint64_t* full() { return (uint64_t*)(ds_smem + bar_off); }
    __device__ static __forceinline__ uint64_t* empty() { return (uint64_t*)(ds_smem + bar_off) + S; }
    __device__ static __forceinline__ uint64_t* never() { return (uint64_t*)(ds_smem + bar_off) + 2 * S; }
    __device__ static __forceinline__ int* abort_flag() { return (int*)(ds_smem + flag_off); }
    __device__ static __forceinline__ int* pending(int warp) { return (int*)(ds_smem + flag_off) + 1 + warp; }
    __device__ static __forceinline__ TC* ow() { return (TC*)(ds_smem + ow_off); }
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
// Interior path: D4 orbit sums of one known slice around the thread's four
// pixels (orbits {same max(|dx|,|dy|), min(|dx|,|dy|)}: 1, 3, 6 for r = 0, 1, 2),
// computed once per slice and kept in registers for both gaps the slice
// brackets; then one weight per orbit and target.
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

template <int R> struct DsNO { static constexpr int N = R == 0 ? 1 : (R == 1 ? 3 : 6); };
template <int GM1> struct DsGP { static constexpr int N = GM1 > 0 ? GM1 : 1; };  // accumulators per pixel

template <typename TI, int R>
__device__ __forceinline__ void ds_orbits(const TI* slot, int lrow, int lcol,
                                          typename DsTypes<TI>::TC (&orb)[KRIG_PX][DsNO<R>::N])
{
    typedef typename DsTypes<TI>::TC TC;
    constexpr int PAD = DsTypes<TI>::PAD, RP = DsTypes<TI>::RP;
    // columns 4-R .. 7+R of the 12 loaded around the thread's four pixels
    TC c0[12], a1[12], a2[12];
    {
        const TI* rowp = slot + (lrow + R) * RP + PAD + lcol;
        TC a[4], b[4], c[4];
        if (R > 0) ld4(rowp - 4, a);
        ld4(rowp, b);
        if (R > 0) ld4(rowp + 4, c);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            c0[q] = R > 0 ? a[q] : TC(0);
            c0[4 + q] = b[q];
            c0[8 + q] = R > 0 ? c[q] : TC(0);
        }
    }
    if (R >= 1) {
        const TI* rm = slot + (lrow + R - 1) * RP + PAD + lcol;
        const TI* rp = slot + (lrow + R + 1) * RP + PAD + lcol;
        TC a[4], b[4], c[4], d[4], e[4], f[4];
        ld4(rm - 4, a);
        ld4(rm, b);
        ld4(rm + 4, c);
        ld4(rp - 4, d);
        ld4(rp, e);
        ld4(rp + 4, f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a1[q] = a[q] + d[q];
            a1[4 + q] = b[q] + e[q];
            a1[8 + q] = c[q] + f[q];
        }
    }
    if (R >= 2) {
        const TI* rm = slot + (lrow + R - 2) * RP + PAD + lcol;
        const TI* rp = slot + (lrow + R + 2) * RP + PAD + lcol;
        TC a[4], b[4], c[4], d[4], e[4], f[4];
        ld4(rm - 4, a);
        ld4(rm, b);
        ld4(rm + 4, c);
        ld4(rp - 4, d);
        ld4(rp, e);
        ld4(rp + 4, f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a2[q] = a[q] + d[q];
            a2[4 + q] = b[q] + e[q];
            a2[8 + q] = c[q] + f[q];
        }
    }
#pragma unroll
    for (int p = 0; p < KRIG_PX; ++p) {
        const int m = 4 + p;  // centre column
        orb[p][0] = c0[m];
        if (R >= 1) {
            orb[p][1] = (c0[m - 1] + c0[m + 1]) + a1[m];
            orb[p][2] = a1[m - 1] + a1[m + 1];
        }
        if (R >= 2) {
            orb[p][3] = (c0[m - 2] + c0[m + 2]) + a2[m];
            orb[p][4] = (a1[m - 2] + a1[m + 2]) + (a2[m - 1] + a2[m + 1]);
            orb[p][5] = a2[m - 2] + a2[m + 2];
        }
    }
}

// The thread's four pixel values of one known slice (the orbit-0 sums).
template <typename TI, int R>
__device__ __forceinline__ void ds_centres(const TI* slot, int lrow, int lcol,
                                           typename DsTypes<TI>::TC (&orb)[KRIG_PX][DsNO<R>::N])
{
    typedef typename DsTypes<TI>::TC TC;
    constexpr int PAD = DsTypes<TI>::PAD, RP = DsTypes<TI>::RP;
    TC b[4];
    ld4(slot + (lrow + R) * RP + PAD + lcol, b);
#pragma unroll
    for (int p = 0; p < KRIG_PX; ++p) {
        orb[p][0] = b[p];
#pragma unroll
        for (int o = 1; o < DsNO<R>::N; ++o) orb[p][o] = TC(0);
    }
}

// Targets t0 and t0 + 1 (t0 + 1 < GM1 or not) of the four pixels from the orbit
// sums of both slices: acc[p][i] = sum_o wl[o][t0+i] lo[p][o] + wh[o][t0+i] hi[p][o];
// ow: the item's [2][NORB][8] orbit weights in shared memory.  One target pair
// at a time keeps few accumulators live beside the two slices' orbit sums.
template <typename TI, int R, int GM1>
__device__ __forceinline__ void ds_fma_pair(typename DsTypes<TI>::TC (&acc)[KRIG_PX][2], int t0,
                                            const typename DsTypes<TI>::TC (&lo)[KRIG_PX][DsNO<R>::N],
                                            const typename DsTypes<TI>::TC (&hi)[KRIG_PX][DsNO<R>::N],
                                            const typename DsTypes<TI>::TC* ow)
{
    typedef typename DsTypes<TI>::TC TC;
    const bool two = t0 + 1 < GM1;
#pragma unroll
    for (int p = 0; p < KRIG_PX; ++p) acc[p][0] = acc[p][1] = TC(0);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int o = 0; o < DsNO<R>::N; ++o) {
            const TC* wp = ow + (s * KRIG_NORB + o) * KRIG_TSLOTS + t0;
            if constexpr (sizeof(TC) == 4) {
                // two targets per packed FMA (fma.rn.f32x2: each half rounds as fmaf)
                const float2 w = *(const float2*)wp;
                const unsigned long long wpk = pk2(w.x, w.y);
#pragma unroll
                for (int p = 0; p < KRIG_PX; ++p) {
                    const TC z = s == 0 ? lo[p][o] : hi[p][o];
                    if (two) {
                        unsigned long long a2 = pk2(acc[p][0], acc[p][1]);
                        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a2) : "l"(wpk), "l"(pk2(z, z)));
                        upk2(a2, acc[p][0], acc[p][1]);
                    } else {
                        acc[p][0] = fmaf(w.x, z, acc[p][0]);
                    }
                }
            } else {
                const double2 w = *(const double2*)wp;
#pragma unroll
                for (int p = 0; p < KRIG_PX; ++p) {
                    const TC z = s == 0 ? lo[p][o] : hi[p][o];
                    acc[p][0] = fma(w.x, z, acc[p][0]);
                    if (two) acc[p][1] = fma(w.y, z, acc[p][1]);
                }
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

// Known slice -> its output slice, bit-exact (u16: float32(u) * scale).
template <typename TI, int R>
__device__ __forceinline__ void ds_passthrough(const DsCtx<TI>& c, int64_t off,
                                               const typename DsTypes<TI>::TC (&orb)[KRIG_PX][DsNO<R>::N])
{
    typedef typename DsTypes<TI>::TO TO;
    TO kv[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) kv[p] = sizeof(TI) == 2 ? (TO)__fmul_rn((float)orb[p][0], c.scale) : (TO)orb[p][0];
    st4<TO>(c.out + off, kv, c.vec_out, c.nvalid);
    if (c.var) {
        const float z4[4] = {0.f, 0.f, 0.f, 0.f};
        st4<float>(c.var + off, z4, c.vec_out, c.nvalid);
    }
}

// Interpolated output slice t (1 <= t < g) of gap j for the interior pixels of
// the four (and their kriging variance).
template <typename TI>
__device__ __forceinline__ void ds_store_t(const DsCtx<TI>& c, int64_t jg, int t, const typename DsTypes<TI>::TC (&acc)[KRIG_PX][2],
                                           int i)
{
    typedef typename DsTypes<TI>::TO TO;
    const int64_t off = jg + (int64_t)t * c.plane;
    if (c.full) {
        TO o[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) o[p] = (TO)acc[p][i];
        st4<TO>(c.out + off, o, true, 4);
    } else {
#pragma unroll
        for (int p = 0; p < 4; ++p)
            if (p >= c.plo && p < c.phi) c.out[off + p] = (TO)acc[p][i];
    }
    if (c.var) {
        const float vv = c.vt[t - 1];
        if (c.full) {
            const float v4[4] = {vv, vv, vv, vv};
            st4<float>(c.var + off, v4, true, 4);
        } else {
            for (int p = c.plo; p < c.phi; ++p) c.var[off + p] = vv;
        }
    }
}

// One item for one consumer warp: its 8 x 16 pixel block of the tile, every
// gap of the item's chunk.  Each known slice's orbit sums are computed once,
// right after its slot fills, and the slot is released at once (the sums stay
// in registers for the next gap).  dry: warm-up pass over the first gap, no
// stores and no release (the slots stay full for the real pass).  Returns
// false if a wait gave up.
// Where the previous slice's orbit sums wait for the next gap: in registers,
// or, for the larger windows (r = 2; r >= 1 in FP64), in the thread's own
// shared-memory rows, so that they are not live while the next slice's sums are
// formed (the consumer code is held to 96 registers).
template <typename TI, int R> struct DsLoSmem { static constexpr bool V = R == 2 || (sizeof(TI) == 8 && R >= 1); };

template <typename TC, int NO>
__device__ __forceinline__ void ds_put_orbits(TC* base, const TC (&o)[KRIG_PX][NO])
{
#pragma unroll
    for (int k = 0; k < NO; ++k) {
        TC* p = base + (size_t)k * (DS_CONSUMERS * 32 * KRIG_PX);
        if constexpr (sizeof(TC) == 4) {
            *(float4*)p = make_float4(o[0][k], o[1][k], o[2][k], o[3][k]);
        } else {
            *(double2*)p = make_double2(o[0][k], o[1][k]);
            *(double2*)(p + 2) = make_double2(o[2][k], o[3][k]);
        }
    }
}

template <typename TC, int NO>
__device__ __forceinline__ void ds_get_orbits(const TC* base, TC (&o)[KRIG_PX][NO])
{
#pragma unroll
    for (int k = 0; k < NO; ++k) {
        TC v[4];
        ld4(base + (size_t)k * (DS_CONSUMERS * 32 * KRIG_PX), v);
#pragma unroll
        for (int p = 0; p < KRIG_PX; ++p) o[p][k] = v[p];
    }
}

// One item for one consumer warp: its 8 x 16 pixel block of the tile, every
// gap of the item's chunk.  Each known slice's orbit sums are computed once,
// right after its slot fills, and the slot is released at once (the sums are
// kept for the next gap).  dry: warm-up pass over the first gap, no stores and
// no release (the slots stay full for the real pass).  Returns false if a wait
// gave up.
template <typename TI, int R, int GM1>
__device__ __forceinline__ bool ds_item(const DsCtx<TI>& c, const DsItem& d, int q, int lrow, int lcol, int lane,
                                        const typename DsTypes<TI>::TC* ow, int nv, bool dry)
{
    typedef typename DsTypes<TI>::TC TC;
    constexpr int S = DsStages<TI>::S;
    constexpr int NO = DsNO<R>::N;
    constexpr bool LS = DsLoSmem<TI, R>::V;
    TI* slots = DsLayout<TI>::slots();
    uint64_t* full = DsLayout<TI>::full();
    uint64_t* empty = DsLayout<TI>::empty();
    constexpr int stride = DsLayout<TI>::stride;
    TC* lsm = DsLayout<TI>::orb(nv) + threadIdx.x * KRIG_PX;  // this thread's rows (consumers: tid < 256)
    const int nsl = dry ? 2 : d.c1 - d.c0 + 1;  // warm-up: the first gap only
    const bool orbits = GM1 > 0 && c.inner;
    TC lo[KRIG_PX][NO];
    if (!mbar_wait(&full[q % S], (q / S) & 1, DS_WAIT_LIMIT)) return false;
    if (orbits) ds_orbits<TI, R>(slots + (q % S) * stride, lrow, lcol, lo);
    else ds_centres<TI, R>(slots + (q % S) * stride, lrow, lcol, lo);
    __syncwarp();
    if (lane == 0 && !dry) mbar_arrive(&empty[q % S]);
    if (LS) ds_put_orbits<TC, NO>(lsm, lo);
    for (int m = 0; m + 1 < nsl; ++m) {
        const int j = d.c0 + m, qh = q + m + 1;
        const int64_t jg = (int64_t)j * c.g * c.plane;
        TC hi[KRIG_PX][NO];
        if (!mbar_wait(&full[qh % S], (qh / S) & 1, DS_WAIT_LIMIT)) return false;
        if (orbits) ds_orbits<TI, R>(slots + (qh % S) * stride, lrow, lcol, hi);
        else ds_centres<TI, R>(slots + (qh % S) * stride, lrow, lcol, hi);
        __syncwarp();
        if (lane == 0 && !dry) mbar_arrive(&empty[qh % S]);
        if (LS) ds_get_orbits<TC, NO>(lsm, lo);
        if (c.mine && !dry) ds_passthrough<TI, R>(c, jg, lo);
        if constexpr (GM1 > 0) {
            if (orbits) {
                // one target pair at a time: the accumulators and weights of one
                // pair live beside the two slices' orbit sums
#pragma unroll
                for (int t0 = 0; t0 < GM1; t0 += 2) {
                    TC acc[KRIG_PX][2];
                    ds_fma_pair<TI, R, GM1>(acc, t0, lo, hi, ow);
                    if (c.clamp) {
#pragma unroll
                        for (int p = 0; p < KRIG_PX; ++p)
#pragma unroll
                            for (int i = 0; i < 2; ++i)  // comparisons keep a NaN (singular system) a NaN
                                acc[p][i] = acc[p][i] < c.lo ? c.lo : (acc[p][i] > c.hi ? c.hi : acc[p][i]);
                    }
                    if (!dry) {
                        ds_store_t<TI>(c, jg, t0 + 1, acc, 0);
                        if (t0 + 1 < GM1) ds_store_t<TI>(c, jg, t0 + 2, acc, 1);
                    }
                }
            }
        }
        if (j == c.jlast && c.mine && !dry) ds_passthrough<TI, R>(c, jg + (int64_t)c.g * c.plane, hi);
        if (LS) {
            ds_put_orbits<TC, NO>(lsm, hi);
        } else {
#pragma unroll
            for (int p = 0; p < KRIG_PX; ++p)
#pragma unroll
                for (int o = 0; o < NO; ++o) lo[p][o] = hi[p][o];
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
    TC* owsm = DsLayout<TI>::ow();
    const DsVolS* tab = DsLayout<TI>::vols(nv);
    constexpr int NW = 2 * KRIG_NORB * KRIG_TSLOTS;
    for (int e = threadIdx.x; e < nv * NW; e += DS_CONSUMERS * 32) {
        const DsVolS& Vv = tab[e / NW];
        owsm[e] = (Vv.dtype == dtype && Vv.cint >= 0) ? ((const TC*)(ws + Vv.otab_off))[e % NW] : TC(0);
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
        const TC* ow = DsLayout<TI>::ow() + v * (2 * KRIG_NORB * KRIG_TSLOTS);
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
            if (!ds_item<TI, R, GM1>(c, d, q, lrow, lcol, a.lane, ow, a.nv, dry)) return -1;
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
