// krig_ds_apply.cuh -- stencil apply of the deduplicated-stencil (DS) form.
//
// Every missing voxel (x, y, jg+t) is the weighted sum of the (2r+1)^2
// windows around (x, y) in known slices j and j+1 (Sec. 4.1.2), with the
// weights of its truncation class solved by k_ds_solve.  k_ds_apply walks the
// work items of Algorithm 1: an item is one 64 x 16 in-plane tile of a run of
// consecutive gaps ("chunk") inside one Z sub-block.  The item's known slices
// (tile plus halo) stream through a ring of shared-memory slots filled by the
// TMA bulk-copy engine (cp.async.bulk, completion on an mbarrier), one slice
// ahead of the compute, so each known slice of the chunk is read from memory
// once.  The item writes its output slices -- the bit-exact copy of its known
// slices (Algorithm 1 step 3) and the interpolated ones -- straight to their
// final offsets (the merge of Sec. 4.2).
//
// Interior pixels (full window) use the D4 symmetry of the interior class:
// the taps of each orbit {same max(|dx|,|dy|), min(|dx|,|dy|)} share one
// weight, so the stencil is applied to orbit sums (6 per slice for r = 2)
// instead of 25 taps.  Pixels within r of the slice border take the general
// path with the full weight row of their own class.  A warp covers a 16 x 8
// block of pixels (four per thread), so only warps at the border diverge.
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
#define DS_FRAMER (DS_CONSUMERS + 1)        // border pixels (frame units)
#define DS_BLOCK ((DS_CONSUMERS + 2) * 32)
#define DS_WAIT_LIMIT (1u << 22)

// Ring depth per input type: enough slots that the producer runs many slices
// ahead of the consumers (a DRAM round trip spans many short gaps), while the
// ring plus the orbit-weight table of all volumes (24 KB, 48 KB for f64)
// stays within about 100 KB of shared memory, so two blocks fit on an SM.
template <typename TI> struct DsStages;
template <> struct DsStages<uint16_t> { static constexpr int S = 16; };
template <> struct DsStages<float> { static constexpr int S = 12; };
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
// Accumulation
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
template <int GM1> struct DsGP { static constexpr int N = GM1 > 0 ? GM1 : 1; };  // accumulators per pixel

// Interior path: orbit sums of each slice times the interior orbit weights.
// ow: shared [2][KRIG_NORB][8] orbit weights.
template <typename TI, int R, int GM1>
__device__ __forceinline__ void ds_accum_interior(typename DsTypes<TI>::TC (&acc)[KRIG_PX][DsGP<GM1>::N],
                                                  const TI* lo, const TI* hi, int lrow, int lcol,
                                                  const typename DsTypes<TI>::TC* ow)
{
    typedef typename DsTypes<TI>::TC TC;
    constexpr int PAD = DsTypes<TI>::PAD, RP = DsTypes<TI>::RP;
    constexpr int NO = R == 0 ? 1 : (R == 1 ? 3 : 6);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const TI* slot = s == 0 ? lo : hi;
        // columns 4-R .. 7+R of the 12 loaded around the thread's four pixels
        TC c0[12], a1[12], a2[12];
        {
            const TI* rowp = slot + (lrow + R) * RP + PAD + lcol;
            TC a[4], b[4], c[4];
            ld4(rowp - 4, a);
            ld4(rowp, b);
            ld4(rowp + 4, c);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                c0[q] = a[q];
                c0[4 + q] = b[q];
                c0[8 + q] = c[q];
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
        TC orb[KRIG_PX][NO];
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
#pragma unroll
        for (int o = 0; o < NO; ++o) {
            TC w[8];
            ldw8(ow + (s * KRIG_NORB + o) * KRIG_TSLOTS, w);
            if constexpr (sizeof(TC) == 4) {
                // two targets per packed FMA (fma.rn.f32x2: each half rounds as fmaf)
#pragma unroll
                for (int p = 0; p < KRIG_PX; ++p) {
                    const unsigned long long ob = pk2(orb[p][o], orb[p][o]);
#pragma unroll
                    for (int t = 0; t + 1 < GM1; t += 2) {
                        unsigned long long a2 = pk2(acc[p][t], acc[p][t + 1]);
                        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a2) : "l"(pk2(w[t], w[t + 1])), "l"(ob));
                        upk2(a2, acc[p][t], acc[p][t + 1]);
                    }
                    if (GM1 & 1) acc[p][GM1 - 1] = fmaf(w[GM1 - 1], orb[p][o], acc[p][GM1 - 1]);
                }
            } else {
#pragma unroll
                for (int p = 0; p < KRIG_PX; ++p)
#pragma unroll
                    for (int t = 0; t < GM1; ++t) acc[p][t] = fma(w[t], orb[p][o], acc[p][t]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent producer / consumer pipeline
//
// Blocks walk the work items round-robin, shape by shape.  Warp DS_PRODUCER
// streams every known slice the block needs, item after item, into a ring of
// DS_STAGES slots ("full" barrier per slot, completed by the bulk copy), after
// the consumers released the slot's previous slice ("empty" barrier, one
// arrival per consumer warp).  The consumer warps compute gap after gap; they
// never wait on each other.  Warp DS_FRAMER computes the border pixels beside
// them.  Every wait is bounded; a wait that gives up sets the device status
// KRIG_DEV_TIMEOUT and the shared abort flag, and the producer then waits
// (bounded) for the copies it still has in flight.
// ---------------------------------------------------------------------------
struct DsItem {
    int v, x0, y0, c0, c1;
};

// Stencil shape of a volume: (r, g) as r * 8 + g - 1.  A block takes its
// items shape by shape (ascending), round-robin within a shape, so that each
// shape's loop runs in code compiled for that shape alone.
#define DS_NSHAPE ((KRIG_RMAX + 1) * 8)
__device__ __forceinline__ int ds_shape(const KrigVol& V) { return V.r * 8 + V.g - 1; }

__device__ __forceinline__ uint32_t ds_shape_mask(const KrigLaunch& P, int dtype)
{
    uint32_t m = 0;
    for (int v = 0; v < P.n_vols; ++v)
        if (P.vol[v].dtype == dtype) m |= 1u << ds_shape(P.vol[v]);
    return m;
}

__device__ __forceinline__ bool ds_decode(const KrigLaunch& P, int it, int dtype, int shape, DsItem& d)
{
    int v = 0;
    for (int u = 1; u < P.n_vols; ++u)
        if (P.vol[u].item_begin <= it) v = u;
    const KrigVol& V = P.vol[v];
    if (V.dtype != dtype || ds_shape(V) != shape) return false;
    // item = ((sub-block b) * chunks + chunk ch) * tiles + tile, divisions by multiply-high
    const uint32_t local = (uint32_t)(it - (int)V.item_begin);
    const uint32_t rest = krig_udiv(local, V.mdiv_tiles), tile = local - rest * (uint32_t)(V.tiles_x * V.tiles_y);
    const uint32_t bb = krig_udiv(rest, V.mdiv_chunks), ch = rest - bb * (uint32_t)V.chunks;
    const uint32_t ty = krig_udiv(tile, V.mdiv_tx), tx = tile - ty * (uint32_t)V.tiles_x;
    const int b = (int)bb;
    const int a0 = b * V.gq + min(b, V.grm), a1 = (b + 1) * V.gq + min(b + 1, V.grm);
    d.v = v;
    d.c0 = a0 + (int)ch * V.chunk;
    d.c1 = min(d.c0 + V.chunk, a1);
    d.x0 = (int)tx * KRIG_TX;
    d.y0 = (int)ty * KRIG_TY;
    return d.c0 < d.c1;
}

// The fields of one volume that the consumer loop needs, one copy per warp in
// shared memory: read from the kernel parameters once per volume instead of
// once per item (parameter reads that miss the constant cache take a round
// trip to L2), without holding registers across the loop.
template <typename TI>
struct DsVolR {
    int v, match;                 // volume index; its items are of this kernel's type and shape
    int item_begin, tiles_x, tiles, chunks, chunk, gq, grm;
    uint64_t mt, mc, mx;          // multiply-high divisors: tiles, chunks, tiles_x
    int H, W, g, jlast, cint;
    float scale;
    typename DsTypes<TI>::TO* out;
    float* var;
    const float* vt;
};

template <typename TI>
__device__ __forceinline__ DsVolR<TI> ds_volr(const KrigLaunch& P, int v, int dtype, int shape)
{
    typedef typename DsTypes<TI>::TO TO;
    const KrigVol& V = P.vol[v];
    DsVolR<TI> R;
    R.v = v;
    R.match = V.dtype == dtype && ds_shape(V) == shape;
    R.item_begin = (int)V.item_begin;
    R.tiles_x = V.tiles_x;
    R.tiles = V.tiles_x * V.tiles_y;
    R.chunks = V.chunks;
    R.chunk = V.chunk;
    R.gq = V.gq;
    R.grm = V.grm;
    R.mt = V.mdiv_tiles;
    R.mc = V.mdiv_chunks;
    R.mx = V.mdiv_tx;
    R.H = V.H;
    R.W = V.W;
    R.g = V.g;
    R.jlast = V.n - 2;
    R.cint = V.cint;
    R.scale = V.scale;
    R.out = (TO*)P.out[v];
    R.var = P.var[v];
    R.vt = (const float*)(P.ws + V.vtab_off) + (int64_t)max(V.cint, 0) * KRIG_TSLOTS;
    return R;
}

// ds_decode on the register copy.
template <typename TI>
__device__ __forceinline__ bool ds_decode_r(const DsVolR<TI>& R, int it, DsItem& d)
{
    const uint32_t local = (uint32_t)(it - R.item_begin);
    const uint32_t rest = krig_udiv(local, R.mt), tile = local - rest * (uint32_t)R.tiles;
    const uint32_t bb = krig_udiv(rest, R.mc), ch = rest - bb * (uint32_t)R.chunks;
    const uint32_t ty = krig_udiv(tile, R.mx), tx = tile - ty * (uint32_t)R.tiles_x;
    const int b = (int)bb;
    const int a0 = b * R.gq + min(b, R.grm), a1 = (b + 1) * R.gq + min(b + 1, R.grm);
    d.v = R.v;
    d.c0 = a0 + (int)ch * R.chunk;
    d.c1 = min(d.c0 + R.chunk, a1);
    d.x0 = (int)tx * KRIG_TX;
    d.y0 = (int)ty * KRIG_TY;
    return d.c0 < d.c1;
}

struct DsShared {
    void* ow;          // interior orbit weights of every volume, [v][2][NORB][8]
    uint64_t* full;
    uint64_t* empty;
    uint64_t* never;  // test hook: a barrier nothing completes
    int* abort;
};

// Dynamic shared memory of k_ds_apply: DS_STAGES slots, the full and empty
// barriers, the test barrier, the abort flag, the orbit weights.  Functions
// derive the pointers from the base themselves (nothing goes through the
// stack of a non-inlined call).
extern __shared__ __align__(128) unsigned char ds_smem[];
template <typename TI> struct DsLayout {
    static constexpr int S = DsStages<TI>::S;
    static constexpr int stride = (KRIG_TY + 2 * KRIG_RMAX) * DsTypes<TI>::RP;  // slot stride, elements
    static constexpr size_t bar_off = (size_t)S * stride * sizeof(TI);
    static constexpr size_t ow_bytes =
        (size_t)KRIG_MAX_VOLUMES * 2 * KRIG_NORB * KRIG_TSLOTS * sizeof(typename DsTypes<TI>::TC);
    static constexpr size_t vr_off = (bar_off + (2 * S + 2) * sizeof(uint64_t) + ow_bytes + 15) / 16 * 16;
    static constexpr size_t bytes = vr_off + DS_CONSUMERS * sizeof(DsVolR<TI>);
    __device__ static __forceinline__ DsVolR<TI>* volr(int warp) { return (DsVolR<TI>*)(ds_smem + vr_off) + warp; }
    __device__ static __forceinline__ TI* slots() { return (TI*)ds_smem; }
    __device__ static __forceinline__ DsShared shared()
    {
        uint64_t* bars = (uint64_t*)(ds_smem + bar_off);
        return DsShared{(void*)(bars + 2 * S + 2), bars, bars + S, bars + 2 * S, (int*)(bars + 2 * S + 1)};
    }
};

// Per-item constants of a consumer thread, taken out of the kernel parameters
// once per item: inside the slice loop the barrier waits (asm with a memory
// clobber) would otherwise force every parameter read to be repeated.
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
};

template <typename TI, int R>
__device__ __forceinline__ DsCtx<TI> ds_ctx(const DsVolR<TI>& V, const DsItem& d, int lrow, int lcol, bool dry)
{
    DsCtx<TI> c;
    const int H = V.H, W = V.W;
    const int y = d.y0 + lrow, xb = d.x0 + lcol;
    c.plane = (int64_t)H * W;
    c.g = V.g;
    c.jlast = V.jlast;
    c.scale = V.scale;
    c.nvalid = min(KRIG_PX, W - xb);
    c.mine = y < H && c.nvalid > 0;
    c.vec_out = (W % KRIG_PX == 0) && c.nvalid == KRIG_PX;
    const int64_t pix = c.mine ? (int64_t)y * W + xb : 0;
    c.out = V.out + pix;
    c.var = (dry || !V.var) ? nullptr : V.var + pix;
    c.vt = V.vt;
    // interior pixels of the four: rows y in [R, H-1-R], x in [R, W-1-R]
    c.plo = max(0, R - xb);
    c.phi = min(c.nvalid, W - R - xb);
    c.inner = c.mine && V.cint >= 0 && y >= R && y <= H - 1 - R && c.plo < c.phi;
    c.full = c.vec_out && c.plo == 0 && c.phi == KRIG_PX;
    return c;
}

// One gap of one item for the consumer warps: passthrough of known slice j
// for every pixel, and the g-1 interpolated slices (with variance) for the
// interior pixels, through the orbit sums.  Frame pixels (within r of the
// border) are written by the frame warp instead.
template <typename TI, int R, int GM1>
__device__ __forceinline__ void ds_gap(const DsCtx<TI>& c, int j, const TI* lo, const TI* hi, int lrow, int lcol,
                                       const typename DsTypes<TI>::TC* ow, bool dry)
{
    typedef typename DsTypes<TI>::TC TC;
    typedef typename DsTypes<TI>::TO TO;
    constexpr int PAD = DsTypes<TI>::PAD, RP = DsTypes<TI>::RP;
    if (!c.mine) return;
    const int64_t jg = (int64_t)j * c.g * c.plane;
    {   // known slice j -> output slice j*g, bit-exact
        TO kv[4];
        const TI* cptr = lo + (lrow + R) * RP + PAD + lcol;
#pragma unroll
        for (int p = 0; p < 4; ++p) kv[p] = (TO)cvt_out(cptr[p], c.scale);
        if (!dry) st4<TO>(c.out + jg, kv, c.vec_out, c.nvalid);
        if (c.var) {
            const float z4[4] = {0.f, 0.f, 0.f, 0.f};
            st4<float>(c.var + jg, z4, c.vec_out, c.nvalid);
        }
        if (j == c.jlast) {  // the volume's last known slice
            const TI* ch_ = hi + (lrow + R) * RP + PAD + lcol;
#pragma unroll
            for (int p = 0; p < 4; ++p) kv[p] = (TO)cvt_out(ch_[p], c.scale);
            const int64_t jg1 = jg + (int64_t)c.g * c.plane;
            if (!dry) st4<TO>(c.out + jg1, kv, c.vec_out, c.nvalid);
            if (c.var) {
                const float z4[4] = {0.f, 0.f, 0.f, 0.f};
                st4<float>(c.var + jg1, z4, c.vec_out, c.nvalid);
            }
        }
    }
    if constexpr (GM1 == 0) {
        return;
    } else {
        if (!c.inner) return;  // no interior pixel among the four
        TC acc[KRIG_PX][DsGP<GM1>::N];
#pragma unroll
        for (int p = 0; p < KRIG_PX; ++p)
#pragma unroll
            for (int t = 0; t < DsGP<GM1>::N; ++t) acc[p][t] = TC(0);
        ds_accum_interior<TI, R, GM1>(acc, lo, hi, lrow, lcol, ow);
        if (dry) return;  // warm-up pass: no stores
        // the g-1 output slices of the gap, one branch for the whole set
        if (c.full) {
#pragma unroll
            for (int t = 0; t < GM1; ++t) {
                TO o[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) o[p] = (TO)acc[p][t];
                st4<TO>(c.out + jg + (int64_t)(t + 1) * c.plane, o, true, 4);
            }
        } else {
#pragma unroll
            for (int t = 0; t < GM1; ++t)
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    if (p >= c.plo && p < c.phi) c.out[jg + (int64_t)(t + 1) * c.plane + p] = (TO)acc[p][t];
        }
        if (c.var) {
#pragma unroll
            for (int t = 0; t < GM1; ++t) {
                const float vv = c.vt[t];
                const int64_t off = jg + (int64_t)(t + 1) * c.plane;
                if (c.full) {
                    const float v4[4] = {vv, vv, vv, vv};
                    st4<float>(c.var + off, v4, true, 4);
                } else {
                    for (int p = c.plo; p < c.phi; ++p) c.var[off + p] = vv;
                }
            }
        }
    }
}

// Frame unit: 32 frame pixels of one gap, one lane each, full weight row of
// the pixel's own truncation class; taps read from global memory (L2).
__device__ __forceinline__ void ds_frame_pixel(const KrigVol& V, int f, int* x, int* y)
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

// Branch-free: tap coordinates are clamped into the slice and truncated taps
// carry zero weight in the class row, so all 2(2R+1)^2 loads are independent
// and in flight together.
template <typename TI, int R, int GM1>
__device__ __noinline__ void ds_frame_unit(const KrigLaunch& P, int v, int j, int f0, int lane)
{
    typedef typename DsTypes<TI>::TC TC;
    typedef typename DsTypes<TI>::TO TO;
    constexpr int N2R = 2 * R + 1, NTAP = 2 * N2R * N2R;
    const KrigVol& V = P.vol[v];
    const int f = f0 + lane;
    if (f >= V.n_frame) return;
    int x, y;
    ds_frame_pixel(V, f, &x, &y);
    const int W = V.W, H = V.H, g = V.g;
    const int64_t plane = (int64_t)H * W;
    const int cy = V.ymap[krig_slot(y, H, R)], cx = V.xmap[krig_slot(x, W, R)];
    const TC* wrow = (const TC*)(P.ws + V.wtab_off) + ((int64_t)cy * V.ncx + cx) * NTAP * KRIG_TSLOTS;
    const TI* in = (const TI*)P.in[v] + (size_t)j * plane;
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
        ldgw8(wrow + k * KRIG_TSLOTS, w);
#pragma unroll
        for (int t = 0; t < GM1; ++t) acc[t] = fma(w[t], z[k], acc[t]);
    }
    TO* out = (TO*)P.out[v];
    float* var = P.var[v];
    const float* vt = (const float*)(P.ws + V.vtab_off) + ((int64_t)cy * V.ncx + cx) * KRIG_TSLOTS;
    const int64_t pix = (int64_t)y * W + x;
#pragma unroll
    for (int t = 0; t < GM1; ++t) {
        out[((int64_t)j * g + t + 1) * plane + pix] = (TO)acc[t];
        if (var) var[((int64_t)j * g + t + 1) * plane + pix] = vt[t];
    }
}

template <typename TI, int GM1>
__device__ __forceinline__ void ds_frame_r(const KrigLaunch& P, int v, int j, int f0, int lane)
{
    switch (P.vol[v].r) {
    case 0: ds_frame_unit<TI, 0, GM1>(P, v, j, f0, lane); break;
    case 1: ds_frame_unit<TI, 1, GM1>(P, v, j, f0, lane); break;
    default: ds_frame_unit<TI, 2, GM1>(P, v, j, f0, lane); break;
    }
}

template <typename TI>
__device__ __forceinline__ void ds_frame_dispatch(const KrigLaunch& P, int v, int j, int f0, int lane)
{
    switch (P.vol[v].g) {
    case 2: ds_frame_r<TI, 1>(P, v, j, f0, lane); break;
    case 3: ds_frame_r<TI, 2>(P, v, j, f0, lane); break;
    case 4: ds_frame_r<TI, 3>(P, v, j, f0, lane); break;
    case 5: ds_frame_r<TI, 4>(P, v, j, f0, lane); break;
    case 6: ds_frame_r<TI, 5>(P, v, j, f0, lane); break;
    case 7: ds_frame_r<TI, 6>(P, v, j, f0, lane); break;
    case 8: ds_frame_r<TI, 7>(P, v, j, f0, lane); break;
    default: break;  // g = 1: nothing to interpolate
    }
}

template <typename TI, int R, int GM1>
__device__ __forceinline__ void ds_consume_item(const KrigLaunch& P, const DsVolR<TI>& VR, const DsItem& d, int q,
                                                TI* slots, int stride, const DsShared& sh, int warp, int lane, bool dry)
{
    constexpr int DS_STAGES = DsStages<TI>::S;
    typedef typename DsTypes<TI>::TC TC;
    // interior orbit weights of the item's volume
    const TC* ow = (const TC*)sh.ow + d.v * (2 * KRIG_NORB * KRIG_TSLOTS);  // shared memory
    const int lrow = (warp >> 2) * 8 + (lane >> 2);
    const int lcol = (warp & 3) * 16 + (lane & 3) * 4;
    const DsCtx<TI> ctx = ds_ctx<TI, R>(VR, d, lrow, lcol, dry);
    const int nsl = dry ? 2 : d.c1 - d.c0 + 1;  // warm-up: the first gap only
    bool ok = mbar_wait(&sh.full[q % DS_STAGES], (q / DS_STAGES) & 1, DS_WAIT_LIMIT);
    for (int m = 0; m + 1 < nsl && ok; ++m) {
        const int ql = q + m, qh = q + m + 1;
        ok = mbar_wait(&sh.full[qh % DS_STAGES], (qh / DS_STAGES) & 1, DS_WAIT_LIMIT);
        if (!ok) break;
        ds_gap<TI, R, GM1>(ctx, d.c0 + m, slots + (ql % DS_STAGES) * stride, slots + (qh % DS_STAGES) * stride, lrow,
                           lcol, ow, dry);
        __syncwarp();
        if (lane == 0 && !dry) mbar_arrive(&sh.empty[ql % DS_STAGES]);
    }
    __syncwarp();
    if (dry) return;  // slots stay full, status untouched
    if (ok) {
        if (lane == 0) mbar_arrive(&sh.empty[(q + nsl - 1) % DS_STAGES]);
    } else {
        if (lane == 0) {
            krig_set_status(P.status, KRIG_DEV_TIMEOUT);
            atomicExch(sh.abort, 1);
        }
    }
}

// All items of one shape for this block, in its order; returns the slice
// sequence number after them.  One non-inlined instance per shape, so the
// call (and its register saves) happens once per block, not once per item.
// dry: warm-up pass over the first gap of the block's first item -- the same
// instructions with no stores and no slot release, run while the class solve
// is still going, so that the code is in the instruction caches when the
// real pass starts (it is cold after the L2 has been flushed).
// The class solve may still be running (programmatic dependent launch): wait
// for it to complete, then copy the interior orbit weights of all volumes,
// now final, into shared memory; a named barrier over the consumer warps only
// (the producer runs on).  Every consumer warp calls this exactly once: before
// its first real item, or after its last shape if it had none.
template <typename TI>
__device__ __noinline__ void ds_weights_ready(const KrigLaunch& P, int dtype)
{
    typedef typename DsTypes<TI>::TC TC;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    TC* owsm = (TC*)DsLayout<TI>::shared().ow;
    const int nv = P.n_vols;
    constexpr int NW = 2 * KRIG_NORB * KRIG_TSLOTS;
    for (int e = threadIdx.x; e < nv * NW; e += DS_CONSUMERS * 32) {
        const KrigVol& Vv = P.vol[e / NW];
        owsm[e] = (Vv.dtype == dtype && Vv.cint >= 0) ? ((const TC*)(P.ws + Vv.otab_off))[e % NW] : TC(0);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(DS_CONSUMERS * 32) : "memory");
}

template <typename TI, int R, int GM1>
__device__ __noinline__ int ds_run_shape(const KrigLaunch& P, int q, int warp, int lane, bool dry, bool* pending)
{
    const int dtype = sizeof(TI) == 8 ? KRIG_F64 : sizeof(TI) == 4 ? KRIG_F32 : KRIG_U16;
    const DsShared sh = DsLayout<TI>::shared();
    const int n_vols = P.n_vols, n_items = (int)P.n_items;
    DsVolR<TI>& VR = *DsLayout<TI>::volr(warp);
    if (lane == 0) VR = ds_volr<TI>(P, 0, dtype, R * 8 + GM1);
    __syncwarp();
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        int v = 0;
        for (int u = 1; u < n_vols; ++u)
            if (P.vol[u].item_begin <= it) v = u;
        if (v != VR.v) {
            __syncwarp();
            if (lane == 0) VR = ds_volr<TI>(P, v, dtype, R * 8 + GM1);
            __syncwarp();
        }
        DsItem d;
        if (!VR.match || !ds_decode_r(VR, it, d)) continue;
        if (*(volatile int*)sh.abort) break;
        // First item of the warp: a warm-up pass over its first gap (same code, no
        // stores) while the class solve may still run, so the consumer code is
        // cached when the weights arrive; only then the wait (ds_weights_ready).
        for (int pass = (!dry && *pending) ? 0 : 1; pass < 2; ++pass) {
            if (pass == 1 && !dry && *pending) {
                ds_weights_ready<TI>(P, dtype);
                *pending = false;
            }
            ds_consume_item<TI, R, GM1>(P, VR, d, q, DsLayout<TI>::slots(), DsLayout<TI>::stride, sh, warp, lane,
                                        dry || pass == 0);
        }
        if (dry) break;
        q += d.c1 - d.c0 + 1;
    }
    return q;
}

template <typename TI, int R>
__device__ __forceinline__ int ds_run_g(int g, const KrigLaunch& P, int q, int warp, int lane, bool dry, bool* pending)
{
    switch (g) {
    case 1: return ds_run_shape<TI, R, 0>(P, q, warp, lane, dry, pending);
    case 2: return ds_run_shape<TI, R, 1>(P, q, warp, lane, dry, pending);
    case 3: return ds_run_shape<TI, R, 2>(P, q, warp, lane, dry, pending);
    case 4: return ds_run_shape<TI, R, 3>(P, q, warp, lane, dry, pending);
    case 5: return ds_run_shape<TI, R, 4>(P, q, warp, lane, dry, pending);
    case 6: return ds_run_shape<TI, R, 5>(P, q, warp, lane, dry, pending);
    case 7: return ds_run_shape<TI, R, 6>(P, q, warp, lane, dry, pending);
    default: return ds_run_shape<TI, R, 7>(P, q, warp, lane, dry, pending);
    }
}

template <typename TI>
__device__ __forceinline__ void ds_produce_slice(const KrigVol& V, const TI* in, const DsItem& d, int s, TI* slot,
                                                 uint64_t* bar, int lane, const CUtensorMap* map)
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
    const TI* src = in + (size_t)s * plane;
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

// One kernel per input type (compiled in separate translation units); items
// of volumes of another type are skipped.
template <typename TI>
__global__ void __launch_bounds__(DS_BLOCK, 2) k_ds_apply(const __grid_constant__ KrigLaunch P,
                                                          const __grid_constant__ DsTma T)
{
    constexpr int DS_STAGES = DsStages<TI>::S;
    constexpr int stride = DsLayout<TI>::stride;
    const int dtype = sizeof(TI) == 8 ? KRIG_F64 : sizeof(TI) == 4 ? KRIG_F32 : KRIG_U16;
    TI* slots = DsLayout<TI>::slots();
    const DsShared sh = DsLayout<TI>::shared();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < DS_STAGES) {
        mbar_init(&sh.full[tid], 1);
        mbar_init(&sh.empty[tid], DS_CONSUMERS);
    }
    if (tid == 0) {
        mbar_init(sh.never, 1);
        *sh.abort = 0;
    }
    fence_proxy_async_smem();
    __syncthreads();
    const int n_items = (int)P.n_items;
    const uint32_t shapes = ds_shape_mask(P, dtype);
    if (warp == DS_PRODUCER) {
        // ---------------- producer warp: the consumers' item order (shape by shape)
        int q = 0;
        bool ok = true;
        for (int it = blockIdx.x, c = 0; c < DS_NSHAPE && ok; it += gridDim.x) {
            if (it >= n_items || !((shapes >> c) & 1u)) {
                ++c;
                it = (int)blockIdx.x - (int)gridDim.x;
                continue;
            }
            DsItem d;
            if (!ds_decode(P, it, dtype, c, d)) continue;
            const KrigVol& V = P.vol[d.v];
            for (int s = d.c0; s <= d.c1; ++s, ++q) {
                const int slot = q % DS_STAGES;
                if (q >= DS_STAGES && !mbar_wait(&sh.empty[slot], ((q / DS_STAGES) - 1) & 1, DS_WAIT_LIMIT)) {
                    ok = false;
                    break;
                }
                if (*(volatile int*)sh.abort) {
                    ok = false;
                    break;
                }
                fence_proxy_async_smem();
                const CUtensorMap* map = (d.v < KRIG_TMA_VOLS && T.valid[d.v]) ? &T.tm[d.v] : nullptr;
                ds_produce_slice<TI>(V, (const TI*)P.in[d.v], d, s, slots + slot * stride, &sh.full[slot], lane, map);
            }
        }
        if (!ok) {
            if (lane == 0) {
                krig_set_status(P.status, KRIG_DEV_TIMEOUT);
                atomicExch(sh.abort, 1);
            }
            // bounded wait for the copies still in flight (the last DS_STAGES issued)
            for (int qq = max(0, q - DS_STAGES); qq < q; ++qq)
                mbar_wait(&sh.full[qq % DS_STAGES], (qq / DS_STAGES) & 1, DS_WAIT_LIMIT);
        }
        return;
    }
    if (warp == DS_FRAMER) {
        // The class solve may still be running (programmatic dependent launch):
        // wait for it to complete before the first read of the weight tables.
        // The producer warp streams input slices only and does not wait; the
        // consumer warps wait in ds_weights_ready.
        asm volatile("griddepcontrol.wait;" ::: "memory");
        // ---------------- frame warp: border pixels (within r of the slice
        // edge, their own truncation classes), latency-bound reads through L2,
        // beside the consumers' tiles
        const int64_t nfu = P.n_frame_units;
        for (int64_t u = blockIdx.x; u < nfu; u += gridDim.x) {
            int v = 0;
            for (int w = 1; w < P.n_vols; ++w)
                if (P.vol[w].frame_begin <= u) v = w;
            const KrigVol& V = P.vol[v];
            if (V.dtype != dtype || V.frame_units == 0) continue;
            const int64_t lu = u - V.frame_begin;
            const int j = (int)(lu / V.frame_units);
            const int f0 = (int)(lu % V.frame_units) * 32;
            ds_frame_dispatch<TI>(P, v, j, f0, lane);
        }
        return;
    }
    // ---------------- consumer warps
    if (P.fault_timeout && blockIdx.x == 0 && warp == 0) {
        // test hook: wait on a barrier nothing completes; the bounded wait gives up
        if (!mbar_wait(sh.never, 0, 1u << 12) && lane == 0) {
            krig_set_status(P.status, KRIG_DEV_TIMEOUT);
            atomicExch(sh.abort, 1);
        }
    }
    int q = 0;
    bool pending = true;  // weights not yet waited for (ds_weights_ready)
    for (int c = 0; c < DS_NSHAPE; ++c) {
        if (!((shapes >> c) & 1u)) continue;
        const int r = c / 8, g = c % 8 + 1;
        if (r == 0) q = ds_run_g<TI, 0>(g, P, q, warp, lane, false, &pending);
        else if (r == 1) q = ds_run_g<TI, 1>(g, P, q, warp, lane, false, &pending);
        else q = ds_run_g<TI, 2>(g, P, q, warp, lane, false, &pending);
    }
    if (pending) ds_weights_ready<TI>(P, dtype);  // no item: still one arrival at the barrier
    (void)slots;
}

template <typename TI>
int krig_launch_ds_apply_t(const KrigLaunch& L, const DsTma& T, cudaStream_t st)
{
    const int dtype = sizeof(TI) == 8 ? KRIG_F64 : sizeof(TI) == 4 ? KRIG_F32 : KRIG_U16;
    bool any = false;
    for (int v = 0; v < L.n_vols; ++v) any = any || L.vol[v].dtype == dtype;
    if (!any) return 0;
    const size_t smem = DsLayout<TI>::bytes;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_ds_apply<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ds_apply<TI>, DS_BLOCK, smem);
    if (e != cudaSuccess) return (int)e;
    const int sms = krig_device_sm_count();
    int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    if (grid > L.n_items) grid = L.n_items;
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
